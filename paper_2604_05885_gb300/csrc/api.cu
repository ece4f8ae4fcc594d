// C ABI entry points (include/jzt.h): argument checks, workspace layout,
// orchestration of the build and walk launchers, status readback.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace jzt {

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int fail_msg(int code, const std::string& msg) { return fail(code, msg); }

static int cuda_fail(cudaError_t e, const char* where) {
  return fail(JZT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int resolve_params(const jzt_params* p, Params* out, const char** why) {
  Params P;
  P.nmax0 = 32;
  P.c = 8;
  P.n_target = 1000;
  P.ngr = 32;
  P.heap = 8;
  P.fac_nodes = 2.0f;
  P.fac_ilist = 128.0f;
  P.reg_fmax = 0.0f;
  P.float_order = 0;
  P.lsd_sort = 0;
  if (p) {
    for (int i = 0; i < 4; ++i)
      if (p->reserved[i] != 0) {
        *why = "jzt_params.reserved must be zero";
        return JZT_ERR_INVALID;
      }
    if (p->nmax0) P.nmax0 = p->nmax0;
    if (p->plane_factor) P.c = p->plane_factor;
    if (p->n_target) P.n_target = p->n_target;
    if (p->ngr) P.ngr = p->ngr;
    if (p->heap_size) P.heap = p->heap_size;
    if (p->alloc_fac_nodes != 0.0f) P.fac_nodes = p->alloc_fac_nodes;
    if (p->alloc_fac_ilist != 0.0f) P.fac_ilist = p->alloc_fac_ilist;
    P.reg_fmax = p->reg_fmax;
    P.float_order = p->float_order;
    P.lsd_sort = p->lsd_sort;
  }
  if (P.lsd_sort != 0 && P.lsd_sort != 1) {
    *why = "lsd_sort must be 0 or 1";
    return JZT_ERR_INVALID;
  }
  if (P.float_order != 0 && P.float_order != 1) {
    *why = "float_order must be 0 or 1";
    return JZT_ERR_INVALID;
  }
  if (P.float_order && P.reg_fmax > 0.0f) {
    *why = "the regularisation (reg_fmax > 0) works on the integer keys only, not with float_order";
    return JZT_ERR_UNSUPPORTED;
  }
  if (!(P.reg_fmax >= 0.0f) || std::isinf(P.reg_fmax)) {
    *why = "reg_fmax must be >= 0 and finite";
    return JZT_ERR_INVALID;
  }
  if (P.nmax0 < 1 || P.nmax0 > 32) { *why = "nmax0 must be in 1..32"; return JZT_ERR_INVALID; }
  if (P.c < 2 || P.c > 64) { *why = "plane_factor must be in 2..64"; return JZT_ERR_INVALID; }
  if (P.n_target < 1) { *why = "n_target must be >= 1"; return JZT_ERR_INVALID; }
  if (P.ngr < 1 || P.ngr > 1024) { *why = "ngr must be in 1..1024"; return JZT_ERR_INVALID; }
  if (P.heap < 2 || P.heap > 16) { *why = "heap_size must be in 2..16"; return JZT_ERR_INVALID; }
  if (!(P.fac_nodes > 0.0f) || !(P.fac_ilist > 0.0f)) {
    *why = "allocation factors must be positive";
    return JZT_ERR_INVALID;
  }
  *out = P;
  return JZT_OK;
}

// Plane 0 always; plane p >= 1 while N / (N_max^(p) / 2) >= N_target.
int num_planes(int64_t n, const Params& P) {
  int p = 1;
  double nmax = P.nmax0;
  while (p < kMaxPlanes) {
    nmax *= P.c;
    if (2.0 * (double)n < (double)P.n_target * nmax) break;
    ++p;
  }
  return p;
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int compute_layout(int64_t n, const Params& P, int k, size_t ws_bytes, Layout* Lp, int64_t n_src) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  L.n = n;
  L.n_src = (n_src >= 0 && n_src < n) ? n_src : n;
  L.nmax0 = P.nmax0;
  L.c = P.c;
  L.n_target = P.n_target;
  L.ngr = P.ngr;
  L.heap = P.heap;
  L.reg_fmax = P.reg_fmax;
  L.float_order = P.float_order;
  L.bucket_sort = (!P.float_order && !P.lsd_sort && n >= kBucketMinN) ? 1 : 0;
  L.fine_bits = 1;  // top F key bits, about 32 points per fine bin on average
  while (L.fine_bits < kMaxFineBits && (n >> (L.fine_bits + 1)) >= 32) ++L.fine_bits;
  L.n_planes = num_planes(n, P);
  // Node capacity per plane: fac * N / (N_max^(p)/2) (Eq. alloc_nodes).  The
  // estimate is not a bound (Sec. II-C), so the small upper planes get 4x the
  // estimate plus slack; never more than the plane below.
  double nmax = P.nmax0;
  for (int p = 0; p < L.n_planes; ++p) {
    double est = std::ceil((double)P.fac_nodes * (double)n / (nmax / 2.0));
    if (p == 0) est = std::max(est, 4096.0);  // small sets: room for mostly tiny leaves
    if (p > 0) est = 4.0 * est + 256.0;
    int64_t cap = (int64_t)std::min<double>(est, (double)n);
    if (p > 0) cap = std::min<int64_t>(cap, L.cap_nodes[p - 1]);
    L.cap_nodes[p] = std::max<int64_t>(cap, 1);
    nmax *= P.c;
  }
  const int64_t cap_sup = (L.cap_nodes[L.n_planes - 1] + P.ngr - 1) / P.ngr;
  L.cap_nodes[L.n_planes] = cap_sup;
  L.n_tiles_sort = (n + kSortTile - 1) / kSortTile;

  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L.meta = take(sizeof(Meta));
  L.keys_a = take(8 * (size_t)n);
  L.keys_b = take(8 * (size_t)n);
  L.vals_a = take(4 * (size_t)n);
  L.vals_b = take(4 * (size_t)n);
  L.lookback = take((size_t)L.n_tiles_sort * kRadixBins * kRadixPasses * 4);
  L.pts = take(16 * (size_t)n);
  if (L.float_order) L.pts_tmp = take(16 * (size_t)n);
  const int64_t scan_tiles = std::max<int64_t>((n + 1 + kScanTile - 1) / kScanTile, 1) + 1;
  L.scan_flags = take(8 * (size_t)scan_tiles);
  for (int p = 0; p <= L.n_planes; ++p) L.spl[p] = take(4 * (size_t)(L.cap_nodes[p] + 1));
  L.gap[0] = L.spl[0];
  for (int p = 1; p < L.n_planes; ++p) L.gap[p] = take(4 * (size_t)(L.cap_nodes[p] + 1));
  for (int p = 0; p < L.n_planes; ++p) L.nsz[p] = take(4 * (size_t)(L.cap_nodes[p] + 1));
  for (int p = 0; p < L.n_planes; ++p) L.nodes[p] = take(sizeof(NodeRec) * (size_t)L.cap_nodes[p]);
  for (int p = 0; p <= L.n_planes; ++p) L.ilo[p] = take(8 * (size_t)L.cap_nodes[p]);
  for (int p = 0; p < L.n_planes; ++p) L.rint[p] = take(4 * (size_t)L.cap_nodes[p]);
  for (int p = 0; p < L.n_planes; ++p) L.ig[p] = take(4 * (size_t)L.cap_nodes[p]);
  for (int p = 0; p < L.n_planes; ++p) L.lk[p] = take((size_t)L.cap_nodes[p]);
  L.ig_pt = take(4 * (size_t)n);
  L.minorig = take(4 * (size_t)n);
  if (L.n_src < n) {
    L.pts2 = take(16 * (size_t)n);
    L.src_pos = take(4 * (size_t)(n + 1));
    L.qrange = take(8 * (size_t)L.cap_nodes[0]);
    L.tile_cnt = take(4 * (size_t)(scan_tiles + 1));
  }
  // Interaction-list arena (Eq. alloc_ilist): fac * N / (N_max^(0)/2) entries,
  // scaled by k/16 for k > 16, plus the dense super-node list; last in the
  // workspace so that a larger workspace simply grows it.
  L.arena = off;
  const int64_t min_entries = cap_sup * cap_sup + 1024;
  if (ws_bytes == 0) {
    const double kfac = std::max(1.0, (double)k / 16.0);
    L.cap_ilist = (int64_t)std::ceil((double)P.fac_ilist * kfac * (double)n / ((double)P.nmax0 / 2.0)) +
                  min_entries;
  } else {
    L.cap_ilist = ws_bytes > off ? (int64_t)((ws_bytes - off) / sizeof(IEntry)) : 0;
  }
  L.cap_ilist = std::min<int64_t>(L.cap_ilist, (int64_t)0xffffffffll);  // 32-bit list offsets
  if (ws_bytes != 0 && L.cap_ilist < min_entries) L.cap_ilist = -1;     // too small
  L.total = align256(L.arena + sizeof(IEntry) * (size_t)std::max<int64_t>(L.cap_ilist, min_entries));
  *Lp = L;
  return JZT_OK;
}

}  // namespace jzt

using namespace jzt;

struct jzt_tree {
  Layout L;
  char* ws;
  int64_t n;      // all points
  int64_t n_src;  // source points (== n for one point set)
  float periodic_L;
};

static int check_n(int64_t n) {
  if (n < 1 || n >= (int64_t(1) << 31))
    return fail(JZT_ERR_INVALID, "N must satisfy 1 <= N < 2^31 (got " + std::to_string(n) + ")");
  return JZT_OK;
}

static int check_L(float L) {
  if (std::isnan(L) || std::isinf(L)) return fail(JZT_ERR_INVALID, "periodic_L must be finite");
  return JZT_OK;
}

extern "C" {

const char* jzt_last_error(void) { return g_err.c_str(); }

const char* jzt_version(void) { return "jzt-gb300 0.1.0 (sm_103a)"; }

int jzt_workspace_bytes(int64_t n, int k_or_0, const jzt_params* p, size_t* bytes) {
  if (!bytes) return fail(JZT_ERR_INVALID, "bytes is null");
  if (int e = check_n(n)) return e;
  if (k_or_0 < 0 || k_or_0 > kMaxKTotal) return fail(JZT_ERR_INVALID, "k_or_0 must be in 0..256");
  Params P;
  const char* why = nullptr;
  if (int e = resolve_params(p, &P, &why)) return fail(e, why);
  Layout L;
  compute_layout(n, P, k_or_0, 0, &L);
  *bytes = L.total;
  return JZT_OK;
}

int jzt_build(const float* d_xyz, int64_t n, float periodic_L, const jzt_params* p, void* d_ws,
              size_t ws_bytes, void* stream, jzt_tree** out) {
  if (!out) return fail(JZT_ERR_INVALID, "out is null");
  *out = nullptr;
  if (!d_xyz || !d_ws) return fail(JZT_ERR_INVALID, "null device pointer");
  if (reinterpret_cast<uintptr_t>(d_xyz) & 3u) return fail(JZT_ERR_INVALID, "d_xyz must be 4-byte aligned");
  if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return fail(JZT_ERR_INVALID, "d_ws must be 256-byte aligned");
  if (int e = check_n(n)) return e;
  if (int e = check_L(periodic_L)) return e;
  Params P;
  const char* why = nullptr;
  if (int e = resolve_params(p, &P, &why)) return fail(e, why);
  Layout L;
  compute_layout(n, P, 0, ws_bytes, &L);
  if (L.cap_ilist < 0) {
    Layout need;
    compute_layout(n, P, 0, 0, &need);
    return fail(JZT_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need.total) +
                                       " bytes, got " + std::to_string(ws_bytes));
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  launch_build(d_xyz, n, periodic_L > 0.0f ? periodic_L : 0.0f, L, static_cast<char*>(d_ws), s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "jzt_build launch");
  jzt_tree* t = new jzt_tree;
  t->L = L;
  t->ws = static_cast<char*>(d_ws);
  t->n = n;
  t->n_src = n;
  t->periodic_L = periodic_L > 0.0f ? periodic_L : 0.0f;
  *out = t;
  return JZT_OK;
}

int jzt_workspace_bytes_query(int64_t n_src, int64_t n_qry, int k, const jzt_params* p, size_t* bytes) {
  if (!bytes) return fail(JZT_ERR_INVALID, "bytes is null");
  if (n_src < 1 || n_qry < 1) return fail(JZT_ERR_INVALID, "need at least one source and one query point");
  if (int e = check_n(n_src + n_qry)) return e;
  if (k < 0 || k > kMaxKTotal) return fail(JZT_ERR_INVALID, "k must be in 0..256");
  Params P;
  const char* why = nullptr;
  if (int e = resolve_params(p, &P, &why)) return fail(e, why);
  Layout L;
  compute_layout(n_src + n_qry, P, k, 0, &L, n_src);
  *bytes = L.total;
  return JZT_OK;
}

int jzt_build_query(const float* d_src, int64_t n_src, const float* d_qry, int64_t n_qry, float periodic_L,
                    const jzt_params* p, void* d_ws, size_t ws_bytes, void* stream, jzt_tree** out) {
  if (!out) return fail(JZT_ERR_INVALID, "out is null");
  *out = nullptr;
  if (!d_src || !d_qry || !d_ws) return fail(JZT_ERR_INVALID, "null device pointer");
  if ((reinterpret_cast<uintptr_t>(d_src) & 3u) || (reinterpret_cast<uintptr_t>(d_qry) & 3u))
    return fail(JZT_ERR_INVALID, "point arrays must be 4-byte aligned");
  if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return fail(JZT_ERR_INVALID, "d_ws must be 256-byte aligned");
  if (n_src < 1 || n_qry < 1) return fail(JZT_ERR_INVALID, "need at least one source and one query point");
  if (int e = check_n(n_src + n_qry)) return e;
  if (int e = check_L(periodic_L)) return e;
  Params P;
  const char* why = nullptr;
  if (int e = resolve_params(p, &P, &why)) return fail(e, why);
  const int64_t n = n_src + n_qry;
  Layout L;
  compute_layout(n, P, 0, ws_bytes, &L, n_src);
  if (L.cap_ilist < 0) {
    Layout need;
    compute_layout(n, P, 0, 0, &need, n_src);
    return fail(JZT_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need.total) +
                                       " bytes, got " + std::to_string(ws_bytes));
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  launch_build_sets(d_src, n_src, d_qry, n_qry, periodic_L > 0.0f ? periodic_L : 0.0f, L, static_cast<char*>(d_ws),
                    s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "jzt_build_query launch");
  jzt_tree* t = new jzt_tree;
  t->L = L;
  t->ws = static_cast<char*>(d_ws);
  t->n = n;
  t->n_src = n_src;
  t->periodic_L = periodic_L > 0.0f ? periodic_L : 0.0f;
  *out = t;
  return JZT_OK;
}

int jzt_tree_knn(jzt_tree* t, int k, int order, int32_t* d_idx, float* d_dist2, void* stream) {
  if (!t) return fail(JZT_ERR_INVALID, "tree is null");
  if (!d_idx || !d_dist2) return fail(JZT_ERR_INVALID, "null output pointer");
  if (k < 1 || (int64_t)k > t->n_src) return fail(JZT_ERR_INVALID, "k must satisfy 1 <= k <= N (sources)");
  if (k > kMaxKTotal) return fail(JZT_ERR_UNSUPPORTED, "k > 256 is not supported");
  if (order != 0 && order != 1) return fail(JZT_ERR_INVALID, "order must be 0 (input) or 1 (z)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  launch_knn(t->L, t->ws, t->periodic_L, k, order, d_idx, d_dist2, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "jzt_tree_knn launch");
  return JZT_OK;
}

int jzt_tree_fof(jzt_tree* t, float b, int32_t* d_labels, void* stream) {
  if (!t) return fail(JZT_ERR_INVALID, "tree is null");
  if (t->n_src < t->n) return fail(JZT_ERR_UNSUPPORTED, "FoF runs on a tree of one point set");
  if (!d_labels) return fail(JZT_ERR_INVALID, "null output pointer");
  if (!(b > 0.0f) || std::isinf(b)) return fail(JZT_ERR_INVALID, "b must be positive and finite");
  if (t->periodic_L > 0.0f && !(b < 0.5f * t->periodic_L))
    return fail(JZT_ERR_INVALID, "periodic boxes need b < L/2");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  launch_fof(t->L, t->ws, t->periodic_L, b, d_labels, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "jzt_tree_fof launch");
  return JZT_OK;
}

int jzt_knn(const float* d_xyz, int64_t n, int k, float periodic_L, int32_t* d_idx, float* d_dist2,
            void* d_ws, size_t ws_bytes, void* stream) {
  if (k < 1 || k > kMaxKTotal || (int64_t)k > n) {
    if (k > kMaxKTotal && (int64_t)k <= n) return fail(JZT_ERR_UNSUPPORTED, "k > 256 is not supported");
    return fail(JZT_ERR_INVALID, "k must satisfy 1 <= k <= N");
  }
  if (!d_idx || !d_dist2) return fail(JZT_ERR_INVALID, "null output pointer");
  jzt_tree* t = nullptr;
  if (int e = jzt_build(d_xyz, n, periodic_L, nullptr, d_ws, ws_bytes, stream, &t)) return e;
  int e = jzt_tree_knn(t, k, 0, d_idx, d_dist2, stream);
  jzt_tree_free(t);
  return e;
}

int jzt_tree_fof_catalogue(jzt_tree* t, float b, const float* d_vel, int min_count, float particle_mass,
                           int32_t* d_labels, int32_t* d_order, jzt_group* d_groups, int64_t cap_groups,
                           int64_t* d_n_groups, void* stream) {
  if (!t) return fail(JZT_ERR_INVALID, "tree is null");
  if (t->n_src < t->n) return fail(JZT_ERR_UNSUPPORTED, "FoF runs on a tree of one point set");
  if (!d_labels || !d_order || !d_n_groups || (cap_groups > 0 && !d_groups))
    return fail(JZT_ERR_INVALID, "null output pointer");
  if (cap_groups < 0) return fail(JZT_ERR_INVALID, "cap_groups must be >= 0");
  if (min_count < 1) return fail(JZT_ERR_INVALID, "min_count must be >= 1");
  if (!std::isfinite(particle_mass)) return fail(JZT_ERR_INVALID, "particle_mass must be finite");
  if (!(b > 0.0f) || std::isinf(b)) return fail(JZT_ERR_INVALID, "b must be positive and finite");
  if (t->periodic_L > 0.0f && !(b < 0.5f * t->periodic_L))
    return fail(JZT_ERR_INVALID, "periodic boxes need b < L/2");
  if (catalogue_scratch_bytes(t->n) > sizeof(IEntry) * (size_t)t->L.cap_ilist)
    return fail(JZT_ERR_WORKSPACE, "workspace too small for the catalogue scratch");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  launch_fof(t->L, t->ws, t->periodic_L, b, d_labels, s);
  if (int e = launch_catalogue(t->L, t->ws, t->periodic_L, d_vel, min_count, particle_mass, d_order, d_groups,
                               cap_groups, d_n_groups, s))
    return e;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "jzt_tree_fof_catalogue launch");
  return JZT_OK;
}

int jzt_selftest_wait(int which, long long limit, void* d_ws, size_t ws_bytes, void* stream, jzt_status_info* info) {
  if (which != 0 && which != 1) return fail(JZT_ERR_INVALID, "which must be 0 (mbarrier) or 1 (flag)");
  if (limit < 1 || limit > (1ll << 26)) return fail(JZT_ERR_INVALID, "limit must be in 1..2^26");
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) return fail(JZT_ERR_INVALID, "bad workspace");
  Params P;
  const char* why = nullptr;
  if (int e = resolve_params(nullptr, &P, &why)) return fail(e, why);
  Layout L;
  compute_layout(1, P, 0, ws_bytes, &L);
  if (L.cap_ilist < 0) return fail(JZT_ERR_WORKSPACE, "workspace too small");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  launch_selftest_wait(L, static_cast<char*>(d_ws), which, limit, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "jzt_selftest_wait launch");
  return jzt_status(d_ws, stream, info);
}

int jzt_knn_query(const float* d_src, int64_t n_src, const float* d_qry, int64_t n_qry, int k, float periodic_L,
                  int32_t* d_idx, float* d_dist2, void* d_ws, size_t ws_bytes, void* stream) {
  if (k < 1 || k > kMaxKTotal || (int64_t)k > n_src) {
    if (k > kMaxKTotal && (int64_t)k <= n_src) return fail(JZT_ERR_UNSUPPORTED, "k > 256 is not supported");
    return fail(JZT_ERR_INVALID, "k must satisfy 1 <= k <= N (sources)");
  }
  if (!d_idx || !d_dist2) return fail(JZT_ERR_INVALID, "null output pointer");
  jzt_tree* t = nullptr;
  if (int e = jzt_build_query(d_src, n_src, d_qry, n_qry, periodic_L, nullptr, d_ws, ws_bytes, stream, &t)) return e;
  int e = jzt_tree_knn(t, k, 0, d_idx, d_dist2, stream);
  jzt_tree_free(t);
  return e;
}

int jzt_fof(const float* d_xyz, int64_t n, float b, float periodic_L, int32_t* d_labels, void* d_ws,
            size_t ws_bytes, void* stream) {
  if (!(b > 0.0f) || std::isinf(b)) return fail(JZT_ERR_INVALID, "b must be positive and finite");
  if (periodic_L > 0.0f && !(b < 0.5f * periodic_L))
    return fail(JZT_ERR_INVALID, "periodic boxes need b < L/2");
  if (!d_labels) return fail(JZT_ERR_INVALID, "null output pointer");
  jzt_tree* t = nullptr;
  if (int e = jzt_build(d_xyz, n, periodic_L, nullptr, d_ws, ws_bytes, stream, &t)) return e;
  int e = jzt_tree_fof(t, b, d_labels, stream);
  jzt_tree_free(t);
  return e;
}

int jzt_status(const void* d_ws, void* stream, jzt_status_info* info) {
  if (!d_ws) return fail(JZT_ERR_INVALID, "d_ws is null");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Meta m;
  cudaError_t e = cudaMemcpyAsync(&m, d_ws, sizeof(Meta), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "jzt_status copy");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "jzt_status synchronize");
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->code = m.status;
    info->detail = m.detail;
    info->required_bytes = m.required_bytes;
    info->ilist_entries = (int64_t)m.arena_peak;
    info->n_planes = m.n_planes;
    info->sort_path = m.bucket_max <= (uint32_t)kGrpStep ? 1 : 0;
    for (int p = 0; p < 16 && p < kMaxPlanes + 1; ++p) info->n_nodes[p] = m.n_nodes[p];
    info->knn_pairs = (int64_t)m.knn_pairs;
    for (int t = 0; t < 8; ++t) info->knn_stats[t] = (int64_t)m.knn_stats[t];
    for (int p = 0; p < 16 && p < kMaxPlanes; ++p) info->knn_plane_entries[p] = (int64_t)m.knn_plane_entries[p];
    info->fof_pairs = (int64_t)m.fof_pairs;
  }
  if (m.status != 0) {
    static const char* names[] = {"ok", "invalid", "unsupported", "cuda", "workspace",
                                  "capacity", "input", "timeout", "internal"};
    int c = -m.status;
    g_err = std::string("device status: ") + (c >= 0 && c < 9 ? names[c] : "?") +
            " (stage " + std::to_string(m.detail) + ")";
  }
  return m.status;
}

int jzt_tree_arrays(const jzt_tree* t, const uint64_t** d_keys, const float** d_pts,
                    int32_t* n_planes) {
  if (!t) return fail(JZT_ERR_INVALID, "tree is null");
  if (d_keys) *d_keys = t->L.float_order ? nullptr : at<uint64_t>(t->ws, t->L.keys_a);
  if (d_pts) *d_pts = at<float>(t->ws, t->L.pts);
  if (n_planes) *n_planes = t->L.n_planes;
  return JZT_OK;
}

int jzt_tree_plane(const jzt_tree* t, int p, int64_t cap, int64_t* n_nodes, int32_t* spl,
                   int32_t* count, float* box, void* stream) {
  if (!t) return fail(JZT_ERR_INVALID, "tree is null");
  if (p < 0 || p >= t->L.n_planes) return fail(JZT_ERR_INVALID, "plane index out of range");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Meta m;
  cudaError_t e = cudaMemcpyAsync(&m, t->ws + t->L.meta, sizeof(Meta), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "jzt_tree_plane");
  const int64_t nn = m.n_nodes[p];
  if (n_nodes) *n_nodes = nn;
  if ((spl || count || box) && cap < nn) return fail(JZT_ERR_INVALID, "buffer capacity below node count");
  if (spl) {
    e = cudaMemcpyAsync(spl, t->ws + t->L.spl[p], 4 * (size_t)(nn + 1), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "jzt_tree_plane spl");
  }
  if (count || box) {
    std::vector<NodeRec> rec((size_t)nn);
    if (nn > 0) {
      e = cudaMemcpyAsync(rec.data(), t->ws + t->L.nodes[p], sizeof(NodeRec) * (size_t)nn,
                          cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return cuda_fail(e, "jzt_tree_plane nodes");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "jzt_tree_plane sync");
    for (int64_t i = 0; i < nn; ++i) {
      if (count) count[i] = rec[i].count;
      if (box) {
        for (int d = 0; d < 3; ++d) {
          box[6 * i + d] = rec[i].lo[d];
          box[6 * i + 3 + d] = rec[i].hi[d];
        }
      }
    }
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "jzt_tree_plane sync");
  return JZT_OK;
}

void jzt_tree_free(jzt_tree* t) { delete t; }

int jzt_profile_enable(int on) { return profile_enable(on); }

int jzt_profile_read(double* ms, int64_t* counts, int n, int64_t* launches) {
  long long l = 0;
  int rc = profile_read(ms, counts, n, &l);
  if (launches) *launches = (int64_t)l;
  return rc ? fail(JZT_ERR_CUDA, "jzt_profile_read: event query failed") : JZT_OK;
}

const char* jzt_profile_phase_name(int i) { return phase_name(i); }

}  // extern "C"
