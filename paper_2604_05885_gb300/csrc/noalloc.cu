// Allocation-free kNN entry point.
//
// Some callers cannot allocate device memory at all: code that runs inside a
// framework which owns every device allocation (and forbids cudaMalloc behind
// its back), or real-time and embedded users that must not enter the allocator
// on their call path.  For them this file provides jzt_knn_noalloc: the same
// build + kNN walk as jzt_knn, with its scratch space taken from one fixed
// device array compiled into the library instead of a caller-provided
// workspace.  The caller still owns the input and output buffers.
//
// The array is g_noalloc_ws below (kNoAllocBytes, 16 MiB).  Every GPU that loads
// the library holds it until the process exits.  In host code its name is only a
// host-side stand-in for the device symbol, so its device address is looked up
// with cudaGetSymbolAddress, once per device and CUDA context, with that device
// current, and that address is what the kernels receive.  The cache is keyed on
// the current context as well, so that after cudaDeviceReset (a new primary
// context, the module loaded again) the address is looked up afresh.  The first
// call on a device (or in a new context) does this set-up and should come before
// any stream capture.
//
// The interaction lists grow with the data (clustered or duplicate-heavy sets
// need longer lists), so even within the size limits a call can run out of the
// fixed array (JZT_ERR_CAPACITY on the device).  The array cannot grow, so no
// retry cures that; such a call fills every output row with index -1 and
// distance NaN, so that a caller who does not read the status cannot mistake
// the rows for results.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "common.cuh"

namespace jzt {

int fail_msg(int code, const std::string& msg);  // api.cu: sets jzt_last_error

namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;  // 16 MiB of scratch per device
constexpr int64_t kNoAllocMaxN = 65536;               // largest N the scratch holds (k <= 32)
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
CUcontext g_ctx[kMaxDevices] = {};
using CtxGetCurrent = CUresult (*)(CUcontext*);
CtxGetCurrent g_get_ctx = nullptr;

// Device address of g_noalloc_ws on the current device, looked up on the first
// call made on that device in its current context (cuCtxGetCurrent is reached
// through the runtime's driver entry point, so the library needs no link to
// the driver library).
int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_msg(JZT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_msg(JZT_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_get_ctx) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail_msg(JZT_ERR_CUDA, "cuCtxGetCurrent is not available from the driver");
    g_get_ctx = reinterpret_cast<CtxGetCurrent>(fn);
  }
  CUcontext ctx = nullptr;  // null before the runtime has set up a context on this thread
  if (g_get_ctx(&ctx) != CUDA_SUCCESS) return fail_msg(JZT_ERR_CUDA, "cuCtxGetCurrent failed");
  if (!ctx || !g_addr[dev] || g_ctx[dev] != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_ws);  // sets up the context if there was none
    if (e != cudaSuccess || !p)
      return fail_msg(JZT_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    if (g_get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return fail_msg(JZT_ERR_CUDA, "no current CUDA context");
    g_addr[dev] = p;
    g_ctx[dev] = ctx;
  }
  *out = g_addr[dev];
  return JZT_OK;
}

// After a failed build or walk (any device-side status), every output entry
// becomes (-1, NaN).
__global__ void k_poison_rows(const Meta* m, int32_t* idx, float* d2, int64_t n_entries) {
  if (*reinterpret_cast<const volatile int32_t*>(&m->status) == 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_entries;
       i += (int64_t)gridDim.x * blockDim.x) {
    idx[i] = -1;
    d2[i] = __int_as_float(0x7fc00000);
  }
}

}  // namespace
}  // namespace jzt

using namespace jzt;

extern "C" int jzt_knn_noalloc(const float* d_xyz, int64_t n, int k, float periodic_L, int32_t* d_idx,
                               float* d_dist2, void* stream, jzt_status_info* info) {
  if (!d_xyz || !d_idx || !d_dist2) return fail_msg(JZT_ERR_INVALID, "null device pointer");
  if (reinterpret_cast<uintptr_t>(d_xyz) & 3u) return fail_msg(JZT_ERR_INVALID, "d_xyz must be 4-byte aligned");
  if (n < 1 || n > kNoAllocMaxN)
    return fail_msg(JZT_ERR_INVALID, "jzt_knn_noalloc handles 1 <= N <= " + std::to_string(kNoAllocMaxN) +
                                         " points (got " + std::to_string(n) + "); use jzt_knn with a workspace");
  if (k < 1 || (int64_t)k > n) return fail_msg(JZT_ERR_INVALID, "k must satisfy 1 <= k <= N");
  if (k > kMaxK) return fail_msg(JZT_ERR_UNSUPPORTED, "k > 32 is not supported");
  if (!std::isfinite(periodic_L)) return fail_msg(JZT_ERR_INVALID, "periodic_L must be finite");
  Params P;
  const char* why = nullptr;
  if (int e = resolve_params(nullptr, &P, &why)) return fail_msg(e, why);
  Layout need;
  compute_layout(n, P, k, 0, &need);
  if (need.total > kNoAllocBytes)
    return fail_msg(JZT_ERR_INVALID, "problem needs " + std::to_string(need.total) + " bytes of scratch, the " +
                                         "built-in array holds " + std::to_string(kNoAllocBytes));
  void* ws = nullptr;
  if (int e = scratch_address(&ws)) return e;
  Layout L;
  compute_layout(n, P, 0, kNoAllocBytes, &L);
  const float pl = periodic_L > 0.0f ? periodic_L : 0.0f;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // Each call starts by re-initialising the status block, counters and look-back
  // tables it uses; nothing else in the array needs to start at zero.
  launch_build(d_xyz, n, pl, L, static_cast<char*>(ws), s);
  launch_knn(L, static_cast<char*>(ws), pl, k, 0, d_idx, d_dist2, s);
  const int64_t entries = n * (int64_t)k;
  k_poison_rows<<<(unsigned)std::min<int64_t>((entries + 255) / 256, 152 * 8), 256, 0, s>>>(
      at<Meta>(static_cast<char*>(ws), L.meta), d_idx, d_dist2, entries);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_msg(JZT_ERR_CUDA, std::string("jzt_knn_noalloc launch: ") + cudaGetErrorString(e));
  if (info) return jzt_status(ws, stream, info);
  return JZT_OK;
}
