// Internal definitions shared by the translation units of libjzt.so:
// the device status/meta block, the workspace layout, and small device helpers
// (sortable float encoding, directed-rounding box distances, bounded waits).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "jzt.h"

namespace jzt {

constexpr int kMaxPlanes = 14;          // planes 0..kMaxPlanes-1, plus the super level
constexpr int kKeyBits = 21;            // per coordinate; 63-bit keys (Sec. II-A)
constexpr int kSentinelLevel = 64;      // level of the gaps before the first / after the last point
constexpr int kIndexLevelOffset = 32;   // equal keys: level = bit_length((i-1)^i) - 32
// LSD radix sort of the 63-bit keys: 8 passes of 8-bit digits (9-bit digits,
// 7 passes, measured slower: twice the digit work per tile and fewer tiles per
// SM).  The digit tables in Meta hold up to kMaxRadixPasses x kMaxRadixBins.
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;                                   // 256
constexpr int kRadixPasses = (3 * kKeyBits + kRadixBits - 1) / kRadixBits;  // 8
constexpr int kMaxRadixPasses = 8;
constexpr int kMaxRadixBins = 512;
constexpr int kSortThreads = 256;
constexpr int kSortIpt = 12;
constexpr int kSortTile = kSortThreads * kSortIpt;  // 3072 keys per radix-sort tile
constexpr int kScanTile = 1024;                      // elements per compaction tile
// Bucket sort of the integer keys (sets of at least kBucketMinN points): one
// scatter into 2^F fine bins (the top F key bits, F <= kMaxFineBits, about 32 to
// 64 points per bin), then a sort of each bin (one warp in registers, or one
// block of kGrpThreads in shared memory for bins of up to kGrpCap keys); taken
// when no bin holds more than kGrpStep keys (else the LSD radix passes run).
constexpr int64_t kBucketMinN = 1 << 16;
constexpr int kMaxFineBits = 24;
constexpr int kGrpThreads = 256;
constexpr int kGrpIpt = 16;
constexpr int kGrpCap = kGrpThreads * kGrpIpt;  // 4096 keys
constexpr int kGrpStep = kGrpCap / 2;
constexpr int kFineScanTile = 4096;             // fine bins per scan tile (256 threads x 16)
constexpr int kMaxK = 32;        // neighbours per LeafToLeaf pass
constexpr int kMaxKTotal = 256;  // neighbours per query (passes of kMaxK; one walk counter each)
constexpr int kCtrLeafSplits = 8;
constexpr int kCtrCoarse = 9;   // + plane
constexpr int kCtrFine = 23;    // fine-bin scan of the bucket sort
constexpr int kCtrN2N = 7;      // kNN NodeToNode parents (walk only: the build's radix passes are done)
constexpr int kCtrLists = 6;    // kNN list sort (walk only, as above)
constexpr int kCtrWalk = 24;
constexpr long long kSpinLimit = 1ll << 22;          // bounded waits (iterations)
constexpr int kCasLimit = 1 << 20;                   // bounded union-find retries

// Stage identifiers stored in Meta::detail on failure.
enum Stage : int32_t {
  kStageNone = 0,
  kStageInput = 1,
  kStageSort = 2,
  kStageSplits = 3,
  kStageNodes = 4,
  kStageTop = 5,
  kStageWalk = 6,
  kStageLeaf = 7,
  kStageFof = 8,
};

// Device-resident status and bookkeeping; lives at offset 0 of the workspace.
// Node-volume classes of the regularisation: 0 = one point (no extent), else
// 1 + 32 + level (volume 2^level; levels -32..63 with the extended equal-key levels).
constexpr int kVolBins = 97;
constexpr int kNoRegLevel = 127;

struct Meta {
  int32_t status;            // jzt_error of the first failure (0 = ok)
  int32_t detail;            // Stage of the first failure
  int64_t required_bytes;    // capacity failures: workspace bytes at least needed
  uint32_t bbox_enc[6];      // sortable-encoded min x,y,z then max x,y,z (open boxes)
  float lo[3];               // quantisation origin
  float scale;               // 2^21 / extent (float32)
  int32_t n_nodes[kMaxPlanes + 1];   // nodes per plane; [n_planes] = super nodes
  uint32_t tile_ctr[32];     // dynamic tile counters: [0,8) radix passes, 8 leaf splits,
                             // 9+p coarse plane p, 24.. walk kernels
  unsigned long long arena_used;     // interaction-list entries handed out
  unsigned long long arena_peak;     // largest arena_used seen this walk
  int32_t n_planes;
  uint32_t bucket_max;               // bucket sort: largest fine-bin count (above kGrpStep: LSD passes)
  uint32_t big_bins;                 // bucket sort: bins left to k_big_bins
  uint32_t big_next;                 // bucket sort: next listed bin to take
  unsigned long long knn_pairs;      // point pairs evaluated by the kNN LeafToLeaf
  unsigned long long knn_stats[8];   // kNN walk statistics (see jzt_status_info)
  unsigned long long knn_plane_entries[kMaxPlanes];  // interaction-list entries per plane
  unsigned long long fof_pairs;      // point pairs evaluated by the FoF LeafToLeaf
  unsigned long long pair_off[kMaxPlanes + 1];  // FoF: pair list of each plane in the arena
  unsigned long long pair_cnt[kMaxPlanes + 1];
  uint32_t radix_offsets[kMaxRadixPasses][kMaxRadixBins];  // exclusive digit offsets per pass
  uint32_t radix_hist[kMaxRadixPasses][kMaxRadixBins];     // digit histograms per pass
  int32_t reg_lvl[kMaxPlanes];       // regularisation: lvl_max per plane (127 = none)
  unsigned long long vol_hist[kVolBins];  // points per node-volume class of one plane
};

// Workspace layout: byte offsets of every sub-buffer (host-computed).
struct Layout {
  int64_t n;
  int32_t nmax0, c, n_target, ngr, heap;
  float reg_fmax;                     // 0: no regularisation
  int32_t float_order;                // 1: float z-order (no keys; pts_tmp is the sort's second buffer)
  int32_t bucket_sort;                // 1: integer keys sorted by fine bins + group sorts (LSD passes as fallback)
  int32_t fine_bits;                  // F: fine bins = the top F key bits
  int32_t n_planes;
  int64_t cap_nodes[kMaxPlanes + 1];  // [n_planes] = super-node capacity
  int64_t cap_ilist;                  // entries
  int64_t n_tiles_sort;
  size_t meta, keys_a, keys_b, vals_a, vals_b, lookback, pts, scan_flags;
  size_t pts_tmp;               // float4 [n] (float order only)
  size_t spl[kMaxPlanes + 1];   // int32 split arrays (cap_nodes+1); [n_planes] = super splits
  size_t gap[kMaxPlanes];       // int32 point-space gap index of each split
  size_t nsz[kMaxPlanes];       // int32 n_i at every split of each plane
  size_t nodes[kMaxPlanes];     // NodeRec per node
  size_t ilo[kMaxPlanes + 1];   // uint2 (offset, count) per receiving node; [n_planes] = supers
  size_t arena;                 // IEntry[cap_ilist]
  size_t rint[kMaxPlanes];      // kNN: float squared internal radius bound per node
  size_t ig[kMaxPlanes];        // FoF: int32 group pointer per node
  size_t lk[kMaxPlanes];        // FoF: uint8 linked flag per node
  size_t ig_pt;                 // FoF: int32 group pointer per sorted point
  size_t minorig;               // FoF: int32 smallest original index per root
  // two point sets (source points first, then query points; Sec. II-G): n_src
  // sources, n - n_src queries; n_src == n for one set
  int64_t n_src;
  size_t pts2;                  // float4 [n]: sources (z order), then queries (z order)
  size_t src_pos;               // int32 [n + 1]: sources before each sorted position
  size_t qrange;                // uint2 per leaf: (first query in the query part, count)
  size_t tile_cnt;              // int32 per scan tile: sources in the tile, then offsets
  size_t total;
};

// 32-byte node record: bounding box, point count, first element.
struct __align__(16) NodeRec {
  float lo[3];
  int32_t count;   // points in the node
  float hi[3];
  int32_t first;   // first point (plane 0) or first child (plane >= 1)
};

// Interaction-list entry (Sec. III-A): source node and the squared lower
// node-node distance r_low^2 (rounded down) used for sorting and early exit.
struct __align__(8) IEntry {
  int32_t src;
  float r2low;
};

// Everything one kNN LeafToLeaf launch needs about one tree (also one job of a
// batch run through the device work queue).
struct L2LArgs {
  const float4* pts;       // source points (sorted; two point sets: the source part)
  const NodeRec* leaves;
  const uint2* ilo;
  const IEntry* arena;
  const float4* qpts;      // query points (== pts for one point set)
  const uint2* qrange;     // per-leaf query ranges (two point sets) or null
  int32_t* out_idx;
  float* out_d2;
  Meta* m;
  int k, k_row, col0, vec_out, order;
  float L;
  int job;                 // index of the job in its batch (queue runs only)
};

struct Params {
  int32_t nmax0, c, n_target, ngr, heap;
  float fac_nodes, fac_ilist;
  float reg_fmax;
  int32_t float_order;  // 1: full-precision float z-order instead of integer keys
  int32_t lsd_sort;     // 1: integer keys always by the LSD radix passes
};

// ---------------------------------------------------------------- host API
int resolve_params(const jzt_params* p, Params* out, const char** why);
int num_planes(int64_t n, const Params& P);
// ws_bytes == 0: size the interaction-list arena for k (jzt_workspace_bytes);
// otherwise the arena takes the whole remainder of a ws_bytes workspace.
// n_src in [0, n): a tree over n_src source points followed by n - n_src query points.
int compute_layout(int64_t n, const Params& P, int k, size_t ws_bytes, Layout* L, int64_t n_src = -1);

// ---------------------------------------------------------------- instrumentation (prof.cu)
enum Phase : int {
  kPhBox = 0, kPhKeys, kPhSort, kPhGather, kPhSplits, kPhNodes,
  kPhKnnTop, kPhKnnN2N, kPhKnnSort, kPhKnnL2L,
  kPhFofTop, kPhFofN2N, kPhFofL2L, kPhFofLabels, kPhaseCount
};
void note_launch(int n = 1);
void prof_begin(int phase, cudaStream_t s);
void prof_end(int phase, cudaStream_t s);
const char* phase_name(int i);
int profile_enable(int on);
int profile_read(double* ms, int64_t* counts, int n, long long* launches);

// ---------------------------------------------------------------- launchers
// build_tree.cu
void launch_build(const float* d_xyz, int64_t n, float periodic_L, const Layout& L,
                  char* ws, cudaStream_t s);
// two point sets: the tree is built over sources then queries (combined index),
// then the sorted points are split by type (sources first) and the leaves get
// per-type ranges; node counts become source counts (Sec. II-G)
void launch_build_sets(const float* d_src, int64_t n_src, const float* d_qry, int64_t n_qry, float periodic_L,
                       const Layout& L, char* ws, cudaStream_t s);
// walk_knn.cu
void launch_knn(const Layout& L, char* ws, float periodic_L, int k, int order, int32_t* d_idx,
                float* d_d2, cudaStream_t s);
// the kNN walk split for batches: everything before the LeafToLeaf on the job's
// own stream, then one persistent LeafToLeaf launch per (k class, boundary)
// over a device queue of (job, leaf) items (kmax: 4, 8, 16 or 32; k <= 32)
void launch_knn_prepare(const Layout& L, char* ws, float periodic_L, int k, cudaStream_t s);
void make_l2l_args(const Layout& L, char* ws, float periodic_L, int k, int32_t* d_idx, float* d_d2, int job,
                   L2LArgs* out);
int queue_kmax(int k);
void launch_put_args(const L2LArgs* h_args, int n, L2LArgs* d_args, cudaStream_t s);
void launch_knn_queue(int kmax, bool periodic, const L2LArgs* d_jobs, int n_jobs, int64_t* d_prefix,
                      unsigned long long* d_next, int32_t* d_job_status, cudaStream_t s);
// walk_fof.cu
void launch_fof(const Layout& L, char* ws, float periodic_L, float b, int32_t* d_labels,
                cudaStream_t s);
// shared (build_tree.cu)
void launch_super_level(const Layout& L, char* ws, cudaStream_t s);
void launch_selftest_wait(const Layout& L, char* ws, int which, long long limit, cudaStream_t s);
size_t catalogue_scratch_bytes(int64_t n);
int launch_catalogue(const Layout& L, char* ws, float periodic_L, const float* d_vel, int min_count,
                     float particle_mass, int32_t* d_order, jzt_group* d_groups, int64_t cap_groups,
                     int64_t* d_n_groups, cudaStream_t s);
void launch_sort_u64(uint64_t* k_a, uint64_t* k_b, uint32_t* v_a, uint32_t* v_b, int64_t n, int passes,
                     uint32_t* lookback, cudaStream_t s, Meta* m);

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ unsigned long long minu64(unsigned long long a, unsigned long long b) {
  return a < b ? a : b;
}

template <typename T>
__host__ __device__ inline T* at(char* ws, size_t off) { return reinterpret_cast<T*>(ws + off); }

// ---------------------------------------------------------------- device helpers
#ifdef __CUDACC__

__device__ __forceinline__ void set_error(Meta* m, int32_t code, int32_t stage) {
  if (atomicCAS(&m->status, 0, code) == 0) m->detail = stage;
}

__device__ __forceinline__ bool failed(const Meta* m) {
  return *reinterpret_cast<const volatile int32_t*>(&m->status) != 0;
}

// Same test, uniform across the warp (lane 0 decides), for kernels that use
// warp collectives after the check.
__device__ __forceinline__ bool warp_failed(const Meta* m) {
  int f = 0;
  if ((threadIdx.x & 31) == 0) f = failed(m) ? 1 : 0;
  return __shfl_sync(0xffffffffu, f, 0) != 0;
}

// Order-preserving map float -> uint32 (total order on non-NaN floats).
__device__ __forceinline__ uint32_t f2sortable(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float sortable2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Relaxed (non-ordering) load at gpu scope: several can be in flight at once.
// Used where the loaded word carries its own flag and value, so no ordering
// with other data is needed.
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Relative slack applied to box-distance bounds so that they stay conservative
// with respect to float32 point distances (each of which carries < 2^-21 error).
constexpr float kLowSlack = 1.0f - 1.0f / 1048576.0f;   // 1 - 2^-20
constexpr float kHighSlack = 1.0f + 1.0f / 1048576.0f;  // 1 + 2^-20

// Per-dimension lower / upper separation of two closed intervals, rounded down /
// up.  Periodic (L > 0): minimum over the images -L, 0, +L for the gap; for the
// span, min over images of the farthest pair, capped at L/2 (minimum image).
__device__ __forceinline__ float gap_rd(float alo, float ahi, float blo, float bhi) {
  return fmaxf(0.0f, fmaxf(__fsub_rd(blo, ahi), __fsub_rd(alo, bhi)));
}
__device__ __forceinline__ float span_ru(float alo, float ahi, float blo, float bhi) {
  return fmaxf(__fsub_ru(bhi, alo), __fsub_ru(ahi, blo));
}
__device__ __forceinline__ float gap_rd_per(float alo, float ahi, float blo, float bhi, float L) {
  float g0 = gap_rd(alo, ahi, blo, bhi);
  float g1 = gap_rd(alo, ahi, __fadd_rd(blo, L), __fadd_ru(bhi, L));
  float g2 = gap_rd(alo, ahi, __fsub_rd(blo, L), __fsub_ru(bhi, L));
  return fminf(g0, fminf(g1, g2));
}
__device__ __forceinline__ float span_ru_per(float alo, float ahi, float blo, float bhi, float L) {
  float s0 = span_ru(alo, ahi, blo, bhi);
  float s1 = span_ru(alo, ahi, __fadd_rd(blo, L), __fadd_ru(bhi, L));
  float s2 = span_ru(alo, ahi, __fsub_rd(blo, L), __fsub_ru(bhi, L));
  return fminf(fminf(s0, fminf(s1, s2)), __fmul_ru(0.5f, L));
}

// Squared lower / upper box-box distances (d_low, d_up of Sec. III-B), as
// conservative float32 bounds.
template <bool PERIODIC>
__device__ __forceinline__ float box_dlow2(const float* alo, const float* ahi, const float* blo,
                                           const float* bhi, float L) {
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float g = PERIODIC ? gap_rd_per(alo[d], ahi[d], blo[d], bhi[d], L)
                       : gap_rd(alo[d], ahi[d], blo[d], bhi[d]);
    s = __fmaf_rd(g, g, s);
  }
  return s * kLowSlack;
}
template <bool PERIODIC>
__device__ __forceinline__ float box_dup2(const float* alo, const float* ahi, const float* blo,
                                          const float* bhi, float L) {
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float g = PERIODIC ? span_ru_per(alo[d], ahi[d], blo[d], bhi[d], L)
                       : span_ru(alo[d], ahi[d], blo[d], bhi[d]);
    s = __fmaf_ru(g, g, s);
  }
  return __fmul_ru(s, kHighSlack);
}

// Union-find on int32 parent pointers that always point to a smaller index
// (so each root is its set's minimum).  Path halving with plain stores is safe:
// a pointer is only ever replaced by one of its own ancestors.
__device__ __forceinline__ int uf_find(int32_t* p, int x) {
  volatile int32_t* vp = p;
  // pointers strictly decrease along a path, so the walk ends; the bound only
  // guards against corrupted input
  for (int it = 0; it < (1 << 26); ++it) {
    int px = vp[x];
    if (px == x) return x;
    int ppx = vp[px];
    if (ppx == px) return px;
    vp[x] = ppx;  // halve the path: ppx is an ancestor of x
    x = ppx;
  }
  return x;
}

// Root of x without writing anything: used where other threads store final
// (contracted) pointers concurrently, which a path-halving store could undo.
__device__ __forceinline__ int uf_root_ro(const int32_t* p, int x) {
  const volatile int32_t* vp = p;
  for (int it = 0; it < (1 << 26); ++it) {
    int px = vp[x];
    if (px == x) return x;
    x = px;
  }
  return x;
}

// Link the sets of a and b (higher root -> lower root) with CAS; returns false if
// the bounded retry budget ran out.
__device__ __forceinline__ bool uf_union(int32_t* p, int a, int b) {
  for (int it = 0; it < kCasLimit; ++it) {
    int ra = uf_find(p, a), rb = uf_find(p, b);
    if (ra == rb) return true;
    int hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
    if (atomicCAS(p + hi, hi, lo) == hi) return true;
  }
  return false;
}

// ---- shared-memory staging by bulk copy (cp.async.bulk) with mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bounded wait on a barrier phase; false when the budget ran out.
// Bounded wait for the phase `parity` of an mbarrier: false after `limit` polls.
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_n(bar, parity, kSpinLimit);
}
// Failure path: wait for a bulk copy this warp issued to land before the warp
// leaves (a CTA must not exit while a copy still writes its shared memory).  The
// copy reads at most 512 bytes of valid device memory, so it completes unless
// the memory system itself has failed; the wait backs off with nanosleep and
// still gives up after about a second rather than hang.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 20); ++it) {
    if (mbar_try_wait(bar, parity)) return;
    __nanosleep(1000);
  }
}

#endif  // __CUDACC__

}  // namespace jzt
