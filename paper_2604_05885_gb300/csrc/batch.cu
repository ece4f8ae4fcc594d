// Batched execution of independent kNN / FoF jobs (no counterpart in the
// paper): each job runs the plain build + walk on one of several lanes
// (streams) with that lane's workspace; lanes fork from and join back to the
// caller's stream through events, so the whole batch is one stream-ordered
// unit that can be captured into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

namespace jzt {

int fail_msg(int code, const std::string& msg);  // api.cu

namespace {

__global__ void k_copy_status(const Meta* m, int32_t* dst) {
  if (threadIdx.x == 0) *dst = m->status;
}

}  // namespace
}  // namespace jzt

using namespace jzt;

namespace {

// Validates every job against the workspace it will run in (ws_of(j), bytes_of(j)).
template <class WsOf, class BytesOf>
int validate_jobs(const jzt_job* jobs, int n_jobs, const Params& P, int n_lanes, WsOf ws_of, BytesOf bytes_of,
                  std::vector<Layout>& lay) {
  lay.assign((size_t)n_jobs, Layout());
  for (int j = 0; j < n_jobs; ++j) {
    const jzt_job& J = jobs[j];
    const std::string tag = "job " + std::to_string(j) + ": ";
    if (!J.d_xyz) return fail_msg(JZT_ERR_INVALID, tag + "null points");
    if (reinterpret_cast<uintptr_t>(J.d_xyz) & 3u) return fail_msg(JZT_ERR_INVALID, tag + "points not 4-byte aligned");
    if (J.n < 1 || J.n >= (int64_t(1) << 31)) return fail_msg(JZT_ERR_INVALID, tag + "N out of range");
    if (!std::isfinite(J.periodic_L)) return fail_msg(JZT_ERR_INVALID, tag + "periodic_L must be finite");
    if (J.lane < 0 || J.lane >= n_lanes) return fail_msg(JZT_ERR_INVALID, tag + "lane out of range");
    if (!ws_of(j) || (reinterpret_cast<uintptr_t>(ws_of(j)) & 255u))
      return fail_msg(JZT_ERR_INVALID, tag + "workspace null or not 256-byte aligned");
    if (J.op == JZT_OP_KNN) {
      if (!J.d_idx || !J.d_dist2) return fail_msg(JZT_ERR_INVALID, tag + "null kNN outputs");
      if (J.k < 1 || (int64_t)J.k > J.n) return fail_msg(JZT_ERR_INVALID, tag + "k must satisfy 1 <= k <= N");
      if (J.k > kMaxKTotal) return fail_msg(JZT_ERR_UNSUPPORTED, tag + "k > 256 is not supported");
    } else if (J.op == JZT_OP_FOF) {
      if (!J.d_labels) return fail_msg(JZT_ERR_INVALID, tag + "null FoF labels");
      if (!(J.b > 0.0f) || std::isinf(J.b)) return fail_msg(JZT_ERR_INVALID, tag + "b must be positive and finite");
      if (J.periodic_L > 0.0f && !(J.b < 0.5f * J.periodic_L))
        return fail_msg(JZT_ERR_INVALID, tag + "periodic boxes need b < L/2");
    } else {
      return fail_msg(JZT_ERR_INVALID, tag + "op must be JZT_OP_KNN or JZT_OP_FOF");
    }
    Params Pj = P;  // the job's own leaf capacity, if it has one
    if (J.nmax0 != 0) {
      if (J.nmax0 < 1 || J.nmax0 > 32) return fail_msg(JZT_ERR_INVALID, tag + "nmax0 must be 0 or in 1..32");
      Pj.nmax0 = J.nmax0;
    }
    compute_layout(J.n, Pj, 0, bytes_of(j), &lay[(size_t)j]);
    if (lay[(size_t)j].cap_ilist < 0) return fail_msg(JZT_ERR_WORKSPACE, tag + "workspace too small");
  }
  return JZT_OK;
}

// Fork: every lane waits for `s0`; join: `s0` waits for every lane.
struct Fork {
  std::vector<cudaEvent_t> ev;
  int open(int n_lanes) {
    ev.assign((size_t)n_lanes + 1, nullptr);
    for (auto& e : ev) {
      cudaError_t ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      if (ce != cudaSuccess) return fail_msg(JZT_ERR_CUDA, std::string("event create: ") + cudaGetErrorString(ce));
    }
    return JZT_OK;
  }
  ~Fork() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

}  // namespace

// Scratch of jzt_batch_run_queue: job descriptors, then per queue class the
// leaf-count prefix (n_jobs + 1 int64) and the queue counter.
constexpr int kQueueClasses = 8;  // kmax 4, 8, 16, 32 x open / periodic

static size_t queue_scratch(int n_jobs, size_t* off_prefix, size_t* off_next) {
  auto a256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t d = a256(sizeof(L2LArgs) * (size_t)(n_jobs > 0 ? n_jobs : 1));
  const size_t pr = a256(sizeof(int64_t) * (size_t)kQueueClasses * (size_t)(n_jobs + 1));
  if (off_prefix) *off_prefix = d;
  if (off_next) *off_next = d + pr;
  return d + pr + a256(sizeof(unsigned long long) * kQueueClasses);
}

extern "C" int jzt_batch_run(const jzt_job* jobs, int n_jobs, const jzt_params* p, void* const* d_lane_ws,
                             const size_t* lane_ws_bytes, void* const* lane_streams, int n_lanes, void* stream,
                             int32_t* d_job_status) {
  if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail_msg(JZT_ERR_INVALID, "jobs is null");
  if (n_lanes < 1 || !d_lane_ws || !lane_ws_bytes || !lane_streams)
    return fail_msg(JZT_ERR_INVALID, "need at least one lane with a workspace and a stream");
  if (!d_job_status && n_jobs > 0) return fail_msg(JZT_ERR_INVALID, "d_job_status is null");
  Params P;
  const char* why = nullptr;
  if (int e = resolve_params(p, &P, &why)) return fail_msg(e, why);
  // validate every job and its lane's workspace before enqueueing anything
  std::vector<Layout> lay;
  if (int e = validate_jobs(jobs, n_jobs, P, n_lanes, [&](int j) { return d_lane_ws[jobs[j].lane]; },
                            [&](int j) { return lane_ws_bytes[jobs[j].lane]; }, lay))
    return e;
  cudaStream_t s0 = reinterpret_cast<cudaStream_t>(stream);
  std::vector<cudaEvent_t> ev((size_t)n_lanes + 1, nullptr);
  for (auto& e : ev) {
    cudaError_t ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      for (auto& x : ev)
        if (x) cudaEventDestroy(x);
      return fail_msg(JZT_ERR_CUDA, std::string("event create: ") + cudaGetErrorString(ce));
    }
  }
  cudaEventRecord(ev[0], s0);
  for (int l = 0; l < n_lanes; ++l) cudaStreamWaitEvent(reinterpret_cast<cudaStream_t>(lane_streams[l]), ev[0], 0);
  for (int j = 0; j < n_jobs; ++j) {
    const jzt_job& J = jobs[j];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(lane_streams[J.lane]);
    char* ws = static_cast<char*>(d_lane_ws[J.lane]);
    const float pl = J.periodic_L > 0.0f ? J.periodic_L : 0.0f;
    const Layout& L = lay[(size_t)j];
    launch_build(J.d_xyz, J.n, pl, L, ws, s);
    if (J.op == JZT_OP_KNN) launch_knn(L, ws, pl, J.k, 0, J.d_idx, J.d_dist2, s);
    else launch_fof(L, ws, pl, J.b, J.d_labels, s);
    k_copy_status<<<1, 32, 0, s>>>(at<Meta>(ws, L.meta), d_job_status + j);
    note_launch();
  }
  for (int l = 0; l < n_lanes; ++l) {
    cudaEventRecord(ev[(size_t)l + 1], reinterpret_cast<cudaStream_t>(lane_streams[l]));
    cudaStreamWaitEvent(s0, ev[(size_t)l + 1], 0);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_msg(JZT_ERR_CUDA, std::string("jzt_batch_run launch: ") + cudaGetErrorString(e));
  return JZT_OK;
}

extern "C" int jzt_batch_queue_bytes(int n_jobs, size_t* bytes) {
  if (!bytes) return fail_msg(JZT_ERR_INVALID, "bytes is null");
  if (n_jobs < 0) return fail_msg(JZT_ERR_INVALID, "n_jobs must be >= 0");
  *bytes = queue_scratch(n_jobs, nullptr, nullptr);
  return JZT_OK;
}

extern "C" int jzt_batch_run_queue(const jzt_job* jobs, int n_jobs, const jzt_params* p, void* const* d_job_ws,
                                   const size_t* job_ws_bytes, void* const* lane_streams, int n_lanes, void* stream,
                                   void* d_scratch, size_t scratch_bytes, int32_t* d_job_status) {
  if (n_jobs < 0 || (n_jobs > 0 && (!jobs || !d_job_ws || !job_ws_bytes)))
    return fail_msg(JZT_ERR_INVALID, "jobs or their workspaces are null");
  if (n_lanes < 1 || !lane_streams) return fail_msg(JZT_ERR_INVALID, "need at least one lane stream");
  if (!d_job_status && n_jobs > 0) return fail_msg(JZT_ERR_INVALID, "d_job_status is null");
  size_t off_prefix = 0, off_next = 0;
  if (!d_scratch || (reinterpret_cast<uintptr_t>(d_scratch) & 255u) ||
      scratch_bytes < queue_scratch(n_jobs, &off_prefix, &off_next))
    return fail_msg(JZT_ERR_WORKSPACE, "scratch null, not 256-byte aligned or smaller than jzt_batch_queue_bytes");
  Params P;
  const char* why = nullptr;
  if (int e = resolve_params(p, &P, &why)) return fail_msg(e, why);
  std::vector<Layout> lay;
  if (int e = validate_jobs(jobs, n_jobs, P, n_lanes, [&](int j) { return d_job_ws[j]; },
                            [&](int j) { return job_ws_bytes[j]; }, lay))
    return e;
  for (int j = 0; j < n_jobs; ++j)
    for (int i = 0; i < j && n_jobs <= 4096; ++i)
      if (d_job_ws[i] == d_job_ws[j])
        return fail_msg(JZT_ERR_INVALID, "job " + std::to_string(j) + ": every job needs a workspace of its own");
  // queued jobs (kNN with k <= 32) in class order: kmax 4, 8, 16, 32, open then periodic
  auto cls_of = [](int k, float L) {
    const int km = queue_kmax(k);
    return (km == 4 ? 0 : km == 8 ? 1 : km == 16 ? 2 : 3) + (L > 0.0f ? 4 : 0);
  };
  std::vector<L2LArgs> args;
  int cls_start[kQueueClasses + 1] = {0};
  for (int c = 0; c < kQueueClasses; ++c) {
    cls_start[c] = (int)args.size();
    for (int j = 0; j < n_jobs; ++j) {
      const jzt_job& J = jobs[j];
      if (J.op != JZT_OP_KNN || J.k > kMaxK || cls_of(J.k, J.periodic_L) != c) continue;
      L2LArgs A;
      make_l2l_args(lay[(size_t)j], static_cast<char*>(d_job_ws[j]), J.periodic_L, J.k, J.d_idx, J.d_dist2, j, &A);
      args.push_back(A);
    }
  }
  cls_start[kQueueClasses] = (int)args.size();
  char* scratch = static_cast<char*>(d_scratch);
  L2LArgs* d_args = reinterpret_cast<L2LArgs*>(scratch);
  int64_t* d_prefix = reinterpret_cast<int64_t*>(scratch + off_prefix);
  unsigned long long* d_next = reinterpret_cast<unsigned long long*>(scratch + off_next);

  cudaStream_t s0 = reinterpret_cast<cudaStream_t>(stream);
  Fork fk;
  if (int e = fk.open(n_lanes)) return e;
  launch_put_args(args.data(), (int)args.size(), d_args, s0);
  cudaEventRecord(fk.ev[0], s0);
  for (int l = 0; l < n_lanes; ++l) cudaStreamWaitEvent(reinterpret_cast<cudaStream_t>(lane_streams[l]), fk.ev[0], 0);
  for (int j = 0; j < n_jobs; ++j) {
    const jzt_job& J = jobs[j];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(lane_streams[J.lane]);
    char* ws = static_cast<char*>(d_job_ws[j]);
    const float pl = J.periodic_L > 0.0f ? J.periodic_L : 0.0f;
    const Layout& L = lay[(size_t)j];
    launch_build(J.d_xyz, J.n, pl, L, ws, s);
    if (J.op == JZT_OP_KNN && J.k <= kMaxK) {
      launch_knn_prepare(L, ws, pl, J.k, s);  // the LeafToLeaf runs from the queue below
      continue;
    }
    if (J.op == JZT_OP_KNN) launch_knn(L, ws, pl, J.k, 0, J.d_idx, J.d_dist2, s);
    else launch_fof(L, ws, pl, J.b, J.d_labels, s);
    k_copy_status<<<1, 32, 0, s>>>(at<Meta>(ws, L.meta), d_job_status + j);
    note_launch();
  }
  for (int l = 0; l < n_lanes; ++l) {
    cudaEventRecord(fk.ev[(size_t)l + 1], reinterpret_cast<cudaStream_t>(lane_streams[l]));
    cudaStreamWaitEvent(s0, fk.ev[(size_t)l + 1], 0);
  }
  for (int c = 0; c < kQueueClasses; ++c) {
    const int n_c = cls_start[c + 1] - cls_start[c];
    if (n_c == 0) continue;
    const int kmax = 4 << (c % 4);
    launch_knn_queue(kmax, c >= 4, d_args + cls_start[c], n_c, d_prefix + (size_t)c * (size_t)(n_jobs + 1),
                     d_next + c, d_job_status, s0);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_msg(JZT_ERR_CUDA, std::string("jzt_batch_run_queue launch: ") + cudaGetErrorString(e));
  return JZT_OK;
}
