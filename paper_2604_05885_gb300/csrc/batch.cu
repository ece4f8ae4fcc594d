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
  std::vector<Layout> lay((size_t)n_jobs);
  for (int j = 0; j < n_jobs; ++j) {
    const jzt_job& J = jobs[j];
    const std::string tag = "job " + std::to_string(j) + ": ";
    if (!J.d_xyz) return fail_msg(JZT_ERR_INVALID, tag + "null points");
    if (reinterpret_cast<uintptr_t>(J.d_xyz) & 3u) return fail_msg(JZT_ERR_INVALID, tag + "points not 4-byte aligned");
    if (J.n < 1 || J.n >= (int64_t(1) << 31)) return fail_msg(JZT_ERR_INVALID, tag + "N out of range");
    if (!std::isfinite(J.periodic_L)) return fail_msg(JZT_ERR_INVALID, tag + "periodic_L must be finite");
    if (J.lane < 0 || J.lane >= n_lanes) return fail_msg(JZT_ERR_INVALID, tag + "lane out of range");
    if (!d_lane_ws[J.lane] || (reinterpret_cast<uintptr_t>(d_lane_ws[J.lane]) & 255u))
      return fail_msg(JZT_ERR_INVALID, tag + "lane workspace null or not 256-byte aligned");
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
    compute_layout(J.n, P, 0, lane_ws_bytes[J.lane], &lay[(size_t)j]);
    if (lay[(size_t)j].cap_ilist < 0) return fail_msg(JZT_ERR_WORKSPACE, tag + "lane workspace too small");
  }
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
