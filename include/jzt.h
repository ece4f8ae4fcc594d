/*
 * jzt.h -- C ABI of the GB300 (sm_103a) jz-tree hot path: exact k-nearest
 * neighbours and friends-of-friends (FoF) groups of 3-D float32 points via a
 * Morton-ordered plane-based tree and a dual tree walk.
 *
 * The method is that of "jz-tree: GPU friendly neighbour search and
 * friends-of-friends with dual tree walks in JAX plus CUDA" (Stuecker, Hahn,
 * Winkler, Gutierrez Adame, Floess; arXiv 2604.05885).  Section references
 * below are to that paper.
 *
 * Conventions for every call:
 *   - Pointers prefixed d_ are DEVICE pointers (cudaMalloc / torch CUDA
 *     storage) on the current device; all others are host pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work is enqueued on it; no call synchronises the
 *     stream unless its comment says so.
 *   - No call allocates device memory.  The caller provides a workspace of at
 *     least jzt_workspace_bytes() bytes (256-byte aligned) and owns it, the
 *     inputs and the outputs.  The library owns only jzt_tree host handles.
 *   - Return codes: JZT_OK on success, else a negative jzt_error value; the
 *     thread-local jzt_last_error() string describes it.  Argument errors are
 *     detected synchronously.  Errors that depend on the data (capacity
 *     overflow, invalid coordinates, exhausted waits) are recorded in a
 *     status word inside the workspace and read with jzt_status().
 *   - Sizes: 1 <= N < 2^31 points.  xyz is N x 3 row-major float32 (x,y,z per
 *     point), 4-byte aligned (16-byte aligned takes the vector-load path).
 *   - periodic_L > 0 selects a periodic box [0,L)^3 with minimum-image
 *     distances (Sec. III-G); every coordinate must lie in [0,L).
 *     periodic_L <= 0 selects open boundaries.
 */
#ifndef JZT_H
#define JZT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum jzt_error {
    JZT_OK = 0,
    JZT_ERR_INVALID = -1,      /* bad argument (N, k, b, L, null pointer, alignment) */
    JZT_ERR_UNSUPPORTED = -2,  /* valid but not implemented here (k > 256; FoF on a query tree) */
    JZT_ERR_CUDA = -3,         /* a CUDA runtime call failed (message in jzt_last_error) */
    JZT_ERR_WORKSPACE = -4,    /* ws_bytes below jzt_workspace_bytes() */
    JZT_ERR_CAPACITY = -5,     /* device: node or interaction-list capacity exceeded */
    JZT_ERR_INPUT = -6,        /* device: NaN/Inf coordinate, or outside [0,L) when periodic */
    JZT_ERR_TIMEOUT = -7,      /* device: a bounded wait or CAS retry loop gave up */
    JZT_ERR_INTERNAL = -8      /* device: an internal consistency check failed (a bug; no
                                  out-of-range access was made) */
} jzt_error;

/* Tree and walk parameters; a zero field takes the default shown. */
typedef struct jzt_params {
    int32_t nmax0;            /* N_max^(0): leaf capacity, 1..32 (default 32; Sec. II-C) */
    int32_t plane_factor;     /* c in N_max^(p) = N_max^(0) c^p (default 8; Sec. II-C) */
    int32_t n_target;         /* coarsening stops below N_target estimated nodes (default 1000) */
    int32_t ngr;              /* NGR: top nodes per super node (default 32; Alg. 1) */
    float alloc_fac_nodes;    /* node capacity per plane = fac * N / (N_max^(p)/2) (default 2; Eq. alloc_nodes) */
    float alloc_fac_ilist;    /* interaction-list capacity = fac * N / (N_max^(0)/2) (default 128; Eq. alloc_ilist) */
    int32_t heap_size;        /* N_r: entries of the FindRmax register heap, 2..16 (default 8; Alg. 3) */
    float reg_fmax;           /* f_max of the plane regularisation (Sec. II-D): 0 = off (default);
                                 > 0: every plane also splits wherever a gap's level exceeds
                                 lvl_max^(p), 2^lvl_max <= f_max V_90% -- results do not change */
    int32_t float_order;      /* 0 (default): 3 x 21-bit integer Morton keys of the quantised points;
                                 1: the full-precision float z-order of Sec. II-A (Eq. msb and its
                                 comparator; Eq. lvl at float32 precision), for data whose scales
                                 span many orders of magnitude -- results do not change, only the
                                 tree; needs 16 more workspace bytes per point; not with reg_fmax */
    int32_t lsd_sort;         /* sort of the integer keys (Sec. II-A, z-order sort; the result is the
                                 same stable order either way): 0 (default) = for N >= 2^16 one
                                 scatter of the keys into fine bins (their top bits) and one sort
                                 per bin (a warp's registers; a block's shared memory above 128
                                 keys), taken when no fine bin holds more than 2048 points and
                                 replaced on the device by the LSD radix passes otherwise;
                                 1 = always the LSD radix passes */
    int32_t reserved[4];      /* must be zero */
} jzt_params;

typedef struct jzt_tree jzt_tree;  /* opaque; lives on the host, points into the workspace */

/* Status block read back by jzt_status. */
typedef struct jzt_status_info {
    int32_t code;             /* jzt_error of the first device-side failure, JZT_OK if none */
    int32_t detail;           /* which stage failed (implementation-defined, for messages) */
    int64_t required_bytes;   /* JZT_ERR_CAPACITY: a workspace size that is at least needed
                                 (a lower bound: later stages may need more) */
    int64_t ilist_entries;    /* interaction-list entries used by the last walk */
    int32_t n_planes;         /* tree-planes built (Sec. II-C) */
    int32_t sort_path;        /* the last build's key sort: 1 = fine-bin bucket sort, 0 = LSD
                                 radix passes (or the float z-order's merge sort) */
    int64_t n_nodes[16];      /* nodes per plane, plane 0 = leaves; [n_planes] = super nodes */
    int64_t knn_pairs;        /* point pairs evaluated by the last kNN LeafToLeaf */
    int64_t fof_pairs;        /* point pairs evaluated by the last FoF LeafToLeaf */
    int64_t knn_stats[8];     /* last kNN LeafToLeaf: [0] list entries examined, [1] source
                                 leaves scanned, [2] candidates queued; [3..7] reserved (0) */
    int64_t knn_plane_entries[16];  /* last kNN walk: interaction-list entries per plane */
} jzt_status_info;

/* Workspace size for N points and parameters p (NULL = defaults).  k_or_0 is the
 * largest k the caller will ask for (0 if only FoF, at most 256): the
 * interaction-list part grows with k above 16.  The interaction-list arena is the last part of the
 * workspace and takes all of it that remains, so a caller that gets
 * JZT_ERR_CAPACITY can retry with a larger workspace (see
 * jzt_status_info.required_bytes) and the same parameters.  Host-only.
 * Errors: JZT_ERR_INVALID for N out of range, bad parameters or null `bytes`. */
int jzt_workspace_bytes(int64_t n, int k_or_0, const jzt_params *p, size_t *bytes);

/* Build the tree of Sec. II on the device: domain (bounding box when open),
 * 3 x 21-bit Morton keys with x most significant (Sec. II-A), stable LSD radix
 * sort of (key, index), gather of the sorted points, gap levels and tree-plane
 * splits (Sec. II-C; N_max^(p) = N_max^(0) c^p), per-node counts and bounding
 * boxes.  d_xyz is read during this call's stream work only: the tree keeps its
 * own sorted copy in the workspace.  *out receives a host handle that stays valid
 * until jzt_tree_free; the workspace must outlive it and must not be reused by
 * another build meanwhile.  Asynchronous; device-side failures go to the status. */
int jzt_build(const float *d_xyz, int64_t n, float periodic_L, const jzt_params *p,
              void *d_ws, size_t ws_bytes, void *stream, jzt_tree **out);

/* Exact k nearest neighbours of every point among all points, the point itself
 * included (Sec. III, Alg. 1-3: dense super-node interaction list, NodeToNode per
 * plane, LeafToLeaf).  Row i of d_idx / d_dist2 (N x k, row-major) lists point i's
 * neighbours by original index, ascending by (float32 squared distance, index).
 * order: 0 = rows in input order (Sec. III-E final reordering), 1 = rows in z order
 * (row r belongs to the point at sorted position r, whose original index is the
 * .w lane of jzt_tree_arrays' pts).  k up to 32 takes one LeafToLeaf pass; larger
 * k (up to 256) takes ceil(k / 32) passes over the same interaction lists, pass j
 * keeping the next 32 keys above the last key of pass j - 1 (the lower radius and
 * index offset of Sec. III-B's repeated LeafToLeaf); the workspace must have been
 * sized for this k (jzt_workspace_bytes), else JZT_ERR_CAPACITY.
 * Errors: JZT_ERR_INVALID (k < 1, k > N, null outputs), JZT_ERR_UNSUPPORTED (k > 256). */
int jzt_tree_knn(jzt_tree *t, int k, int order, int32_t *d_idx, float *d_dist2, void *stream);

/* FoF groups at linking length b (Sec. IV): points i, j are friends when their
 * float32 squared distance is <= b*b (float32); groups are the connected
 * components.  d_labels[i] (N int32, input order) = smallest original index in
 * point i's group.  Whole-node links when the node-node upper distance is <= b
 * (Sec. IV-A).  Errors: JZT_ERR_INVALID (b <= 0 or not finite, periodic b >= L/2). */
int jzt_tree_fof(jzt_tree *t, float b, int32_t *d_labels, void *stream);

/* ---- Separate query and source points (Sec. II-G, multiple point types).
 * One tree is built jointly over the n_src source points followed by the n_qry
 * query points (one combined index for the sort; a node splits while it holds
 * more than N_max^(p) points of both types together, which bounds each type's
 * count as Sec. II-G requires).  After the build the sorted points are separated
 * by type, each in z order, and every leaf gets a source range and a query
 * range; node counts used by the radius search are source counts.
 * jzt_tree_knn on such a tree writes n_qry rows (row r: query r; order 1: query
 * z order) of the k nearest sources (source indices), 1 <= k <= min(256, n_src);
 * jzt_tree_fof returns JZT_ERR_UNSUPPORTED.  Workspace: jzt_workspace_bytes_query.
 * Errors as jzt_build, plus JZT_ERR_INVALID for n_src < 1 or n_qry < 1. */
int jzt_workspace_bytes_query(int64_t n_src, int64_t n_qry, int k, const jzt_params *p, size_t *bytes);
int jzt_build_query(const float *d_src, int64_t n_src, const float *d_qry, int64_t n_qry,
                    float periodic_L, const jzt_params *p, void *d_ws, size_t ws_bytes,
                    void *stream, jzt_tree **out);
/* One call: build over both sets, then kNN of every query point among the sources. */
int jzt_knn_query(const float *d_src, int64_t n_src, const float *d_qry, int64_t n_qry, int k,
                  float periodic_L, int32_t *d_idx, float *d_dist2, void *d_ws, size_t ws_bytes,
                  void *stream);

/* ---- FoF catalogue (Sec. IV-B, catalogue reduction). */
typedef struct jzt_group {
    int32_t label;        /* the group's FoF label (smallest original index) */
    int32_t count;        /* points in the group */
    int64_t offset;       /* position of the group's first point in d_order */
    float mass;           /* count * particle_mass */
    float x_cm[3];        /* centre of mass; periodic: of the minimum-image positions
                             relative to the group's root, wrapped into [0, L) */
    float v_cm[3];        /* centre-of-mass velocity (0 when d_vel is NULL) */
    float r_inertia;      /* sqrt of the mean squared distance to x_cm */
} jzt_group;             /* 48 bytes */

/* FoF at linking length b (as jzt_tree_fof, labels into d_labels), then the
 * catalogue: d_order (N int32) receives the original indices in group order -- a
 * stable sort of the z-ordered points by the z position of their group's root
 * (the member with the lowest z position), so roots keep their z order and every
 * group is a contiguous block in z order -- and d_groups the groups of at least
 * min_count points, in group order, up to cap_groups of them; *d_n_groups
 * (device int64) receives their number.  More than cap_groups groups: the first
 * cap_groups are written and the status reports JZT_ERR_CAPACITY.  Sums are
 * taken in float64 in a fixed order (deterministic).  d_vel: N x 3 float32
 * velocities in input order, or NULL.  Scratch comes from the interaction-list
 * part of the workspace (about 36 bytes per point; JZT_ERR_WORKSPACE if it is
 * smaller).  Errors as jzt_tree_fof, plus JZT_ERR_INVALID (min_count < 1,
 * particle_mass not finite, null outputs, cap_groups < 0) and
 * JZT_ERR_UNSUPPORTED on a query tree. */
int jzt_tree_fof_catalogue(jzt_tree *t, float b, const float *d_vel, int min_count, float particle_mass,
                           int32_t *d_labels, int32_t *d_order, jzt_group *d_groups, int64_t cap_groups,
                           int64_t *d_n_groups, void *stream);

/* One-call forms: build, then walk, on the same workspace. */
int jzt_knn(const float *d_xyz, int64_t n, int k, float periodic_L,
            int32_t *d_idx, float *d_dist2, void *d_ws, size_t ws_bytes, void *stream);
int jzt_fof(const float *d_xyz, int64_t n, float b, float periodic_L,
            int32_t *d_labels, void *d_ws, size_t ws_bytes, void *stream);

/* Synchronises `stream`, then reads the status block of workspace d_ws into *info
 * (may be NULL) and returns its code (JZT_OK or a device-side jzt_error).
 * Returns JZT_ERR_CUDA if the synchronisation itself fails. */
int jzt_status(const void *d_ws, void *stream, jzt_status_info *info);

/* Device pointers into the tree (valid while the tree lives):
 *   keys  -- N uint64 Morton keys, sorted ascending (NULL for a tree built with
 *            float_order = 1, which sorts by the float comparator and has no keys)
 *   pts   -- N float4 sorted points (x, y, z, and in .w the original index of
 *            the point as int32 bits)
 * and the number of planes.  Host-only, no CUDA call. */
int jzt_tree_arrays(const jzt_tree *t, const uint64_t **d_keys, const float **d_pts,
                    int32_t *n_planes);

/* Copies plane p of the tree to HOST buffers (synchronises `stream`):
 *   spl   -- n_nodes+1 int32 splits: point indices for p = 0, indices into plane
 *            p-1's nodes for p >= 1 (Sec. II-C, Fig. tree_construction)
 *   count -- n_nodes int32 points per node
 *   box   -- n_nodes x 6 float32 bounding boxes (lo x,y,z, hi x,y,z)
 * Any of spl/count/box may be NULL.  cap is the capacity (in nodes) of the
 * caller's buffers; *n_nodes receives the node count.
 * Errors: JZT_ERR_INVALID (p out of range, cap too small). */
int jzt_tree_plane(const jzt_tree *t, int p, int64_t cap, int64_t *n_nodes,
                   int32_t *spl, int32_t *count, float *box, void *stream);

void jzt_tree_free(jzt_tree *t);

/* ---- Batched jobs (no counterpart in the paper: a system pattern on top of the
 * method).  Each job is an independent point set with its own operation. */
enum { JZT_OP_KNN = 0, JZT_OP_FOF = 1 };

typedef struct jzt_job {
    const float *d_xyz;   /* N x 3 float32 points (device) */
    int64_t n;            /* 1 <= N < 2^31 */
    float periodic_L;     /* > 0: periodic box [0,L)^3 */
    int32_t op;           /* JZT_OP_KNN or JZT_OP_FOF */
    int32_t k;            /* kNN: neighbours per point, 1..min(256, N) */
    float b;              /* FoF: linking length */
    int32_t lane;         /* lane (0 <= lane < n_lanes) that runs the job */
    int32_t nmax0;        /* this job's leaf capacity N_max^(0), 1..32; 0 = that of the batch's params
                             (results never depend on it; an autotuner picks it per set size) */
    int32_t *d_idx;       /* kNN output, N x k (input order), as jzt_tree_knn */
    float *d_dist2;       /* kNN output, N x k */
    int32_t *d_labels;    /* FoF output, N, as jzt_tree_fof */
} jzt_job;

/* Runs n_jobs jobs: the work of each job is exactly that of jzt_knn / jzt_fof
 * (same results).  Job j runs on lane jobs[j].lane, i.e. on lane_streams[lane]
 * with workspace d_lane_ws[lane] of lane_ws_bytes[lane] bytes (at least
 * jzt_workspace_bytes of every job on that lane, for that job's k); jobs on one
 * lane run in array order and reuse its workspace, lanes run concurrently.  The
 * lanes fork from `stream` and join back into it with events, so the batch is
 * ordered like one operation on `stream` and can be captured into a CUDA graph
 * (capture `stream`; the lane streams join the capture through the events).
 * d_job_status (device, n_jobs int32) receives each job's device status code
 * (JZT_OK or a device-side jzt_error) when the job ends.  All arguments are
 * validated before anything is enqueued (JZT_ERR_INVALID / _UNSUPPORTED /
 * _WORKSPACE with a message naming the job). */
int jzt_batch_run(const jzt_job *jobs, int n_jobs, const jzt_params *p,
                  void *const *d_lane_ws, const size_t *lane_ws_bytes,
                  void *const *lane_streams, int n_lanes, void *stream, int32_t *d_job_status);

/* Batched jobs with the kNN LeafToLeaf of all jobs in persistent launches over a
 * device work queue (no counterpart in the paper).  Same results as jzt_batch_run
 * and as one jzt_knn / jzt_fof call per job.  Every job has a workspace of its own
 * (d_job_ws[j], job_ws_bytes[j] bytes: at least jzt_workspace_bytes of that job;
 * two jobs may not share one) because all the kNN trees must exist at once: each
 * job's build and everything of its walk before the LeafToLeaf run on lane
 * lane_streams[jobs[j].lane] (jobs of one lane in array order, lanes concurrently);
 * then, on `stream`, for each class of kNN jobs with k <= 32 (k rounded up to 4,
 * 8, 16 or 32, open or periodic boundaries) one persistent kernel pops (job, leaf)
 * items from a device queue until every leaf of every job of the class is done.
 * FoF jobs and kNN jobs with k > 32 run entirely on their lanes.  The lanes fork
 * from and join back into `stream` with events, so the batch is one
 * stream-ordered operation that can be captured into a CUDA graph.
 * d_scratch: device memory of at least jzt_batch_queue_bytes(n_jobs) bytes,
 * 256-byte aligned, owned by the caller (the job descriptors, the queues'
 * leaf-count prefixes and counters live there).  d_job_status receives every
 * job's device status code.  All arguments are validated before anything is
 * enqueued (JZT_ERR_INVALID / _UNSUPPORTED / _WORKSPACE, the message naming the
 * job). */
int jzt_batch_queue_bytes(int n_jobs, size_t *bytes);
int jzt_batch_run_queue(const jzt_job *jobs, int n_jobs, const jzt_params *p, void *const *d_job_ws,
                        const size_t *job_ws_bytes, void *const *lane_streams, int n_lanes, void *stream,
                        void *d_scratch, size_t scratch_bytes, int32_t *d_job_status);

/* Allocation-free form of jzt_knn (the paper has no counterpart: this is for
 * callers that may not allocate device memory, e.g. code inside a framework that
 * owns all device allocations, or a real-time path that must not enter the
 * allocator).  Same results as jzt_knn (rows in input order), but the scratch
 * space is a fixed 16 MiB device array inside the library rather than a caller
 * workspace; the caller still owns d_xyz, d_idx and d_dist2.  Limits:
 * 1 <= N <= 65536, 1 <= k <= min(32, N); larger sizes return JZT_ERR_INVALID with
 * a message naming the limit.  Calls no allocator.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current, so make that first call before any stream capture; the address is kept
 * per device and CUDA context, and looked up again when the current context
 * changes (after cudaDeviceReset, for instance).  All calls share the one array per device: calls that overlap
 * on the GPU (on different streams or threads) race and must be serialised by
 * the caller; each call re-initialises what it needs, the rest keeps the
 * previous call's data.
 * The interaction lists grow with the data, so even within the limits a
 * clustered or duplicate-heavy set can run out of the fixed array: a device-side
 * JZT_ERR_CAPACITY that no retry cures (the array cannot grow; use jzt_knn with
 * a workspace of the size jzt_status reports).  After any device-side error
 * every output entry is set to index -1, distance NaN.
 * info: NULL to return after enqueueing the work (device-side errors are then
 * visible only as those -1 / NaN rows); otherwise the call synchronises `stream`
 * and fills *info like jzt_status (device-side errors are then returned as the
 * call's result). */
int jzt_knn_noalloc(const float *d_xyz, int64_t n, int k, float periodic_L,
                    int32_t *d_idx, float *d_dist2, void *stream, jzt_status_info *info);

/* Failure-path self-test (no counterpart in the paper): makes one of the library's
 * bounded waits run out -- which = 0: an mbarrier phase that never completes (the
 * LeafToLeaf staging wait), 1: a published word that nobody sets (the radix-sort
 * look-back poll) -- after `limit` polls (1..2^26), then synchronises `stream` and
 * returns the status like jzt_status: JZT_ERR_TIMEOUT when the wait gave up.  The
 * context stays usable.  d_ws: any workspace of at least jzt_workspace_bytes(1, 0)
 * bytes (its status block is overwritten). */
int jzt_selftest_wait(int which, long long limit, void *d_ws, size_t ws_bytes, void *stream,
                      jzt_status_info *info);

/* Instrumentation (no counterpart in the paper; used to measure the kernels).
 * jzt_profile_enable(1) makes every later call record a CUDA event pair on its
 * own stream around each kernel phase (phase names: jzt_profile_phase_name).
 * jzt_profile_read waits for the recorded events, writes the summed duration
 * in milliseconds and the number of recorded instances of phase i to ms[i] and
 * counts[i] (i < n; either array may be NULL), writes to *launches the number of
 * kernels this library launched since the previous read (counted whether or
 * not profiling is on; may be NULL), and clears the records.  Host-only state,
 * shared by all threads; returns JZT_ERR_CUDA if an event could not be read. */
int jzt_profile_enable(int on);
int jzt_profile_read(double *ms, int64_t *counts, int n, int64_t *launches);
/* Name of phase i, or NULL past the last phase. */
const char *jzt_profile_phase_name(int i);

/* Thread-local description of the last error returned on this thread. */
const char *jzt_last_error(void);

/* Library version string. */
const char *jzt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JZT_H */
