// Dual tree walk for exact k-nearest neighbours (Sec. III, Alg. 1-3).
//
//  * super level: NGR top nodes per super node, dense interaction list (Alg. 1).
//  * NodeToNode per plane (Alg. 2): one warp per receiving parent; G lanes per
//    child split the candidate children.  FindRmax (Alg. 3) keeps a register
//    heap of (d_up^2, count) pairs; Count and Insert then keep the candidates
//    with d_low^2 <= R_max^2.  The three phases are fused in one launch: the
//    warp reserves its output range in the interaction-list arena with one
//    atomic instead of a separate prefix-sum launch.
//  * every receiver's list is sorted by r_low^2 (bitonic, one warp per list) so
//    that walks can stop early (Sec. III-D).
//  * LeafToLeaf: one warp per query leaf, one (or G) lanes per query point; a
//    per-lane register top-k ordered by (float32 d2, original index); candidates
//    that beat the running k-th distance are queued in shared memory and merged
//    in batches so that the warp does not serialise on single insertions.
#include <cuda_runtime.h>

#include <climits>

#include "common.cuh"

namespace jzt {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kUnsortedBit = 0x80000000u;

__device__ __forceinline__ uint32_t warp_incl_scan_u(uint32_t v) {
  const int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// ------------------------------------------------------------------ reset / top level

__global__ void k_walk_reset(Meta* m) {
  if (threadIdx.x == 0) {
    m->arena_used = 0;
    m->arena_peak = 0;
    m->knn_pairs = 0;
  }
  if (threadIdx.x >= kCtrWalk && threadIdx.x < 32) m->tile_ctr[threadIdx.x] = 0;
}

// Dense interaction list over the super nodes (Sec. III-A: ispl_i = N i,
// isrc_j = j mod N), r_low = 0.  upper: FoF keeps only pairs j >= i.
__global__ void k_dense_ilist(const Meta* mc, uint2* ilo_sup, IEntry* arena, int sup_plane,
                              int upper, int64_t cap_ilist, Meta* m) {
  if (failed(mc)) return;
  const int64_t ns = mc->n_nodes[sup_plane];
  const int64_t total = upper ? ns * (ns + 1) / 2 : ns * ns;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (total > cap_ilist) set_error(m, JZT_ERR_CAPACITY, kStageTop);
    m->arena_used = (unsigned long long)total;
  }
  if (total > cap_ilist) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t off = upper ? (i * ns - i * (i - 1) / 2) : i * ns;
    int64_t cnt = upper ? ns - i : ns;
    ilo_sup[i] = make_uint2((uint32_t)off, (uint32_t)cnt);
    for (int64_t j = 0; j < cnt; ++j) {
      IEntry e;
      e.src = (int32_t)(upper ? i + j : j);
      e.r2low = 0.0f;
      arena[off + j] = e;
    }
  }
}

// ------------------------------------------------------------------ FindRmax heap
// Register heap of NR (radius^2, count) pairs sorted by radius (Sec. III-B,
// after the register heaps of Jakob & Guthe).  RadiusOfCount = smallest radius
// whose cumulative count reaches k, +inf if the total is below k.  When the heap
// is full and dropping its largest entry would lose needed count, the new count
// is added to the first entry with a larger radius instead (a conservative
// merge: counts only ever move to larger radii).
template <int NR>
struct RHeap {
  float r[NR];
  int c[NR];
  float rad;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int t = 0; t < NR; ++t) {
      r[t] = INFINITY;
      c[t] = 0;
    }
    rad = INFINITY;
  }
  __device__ __forceinline__ void update_rad(int k) {
    int cum = 0;
    float res = INFINITY;
#pragma unroll
    for (int t = 0; t < NR; ++t) {
      cum += c[t];
      if (cum >= k && res == INFINITY) res = r[t];
    }
    rad = res;
  }
  __device__ __forceinline__ void insert(float rr, int cc, int k) {
    // position = number of entries with radius <= rr
    int pos = 0;
#pragma unroll
    for (int t = 0; t < NR; ++t) pos += (r[t] <= rr) ? 1 : 0;
    int before_last = 0;
#pragma unroll
    for (int t = 0; t < NR - 1; ++t) before_last += c[t];
    const bool can_drop = (c[NR - 1] == 0) || (before_last + (pos < NR ? cc : 0) >= k);
    if (pos == NR) {
      // larger than every stored radius: fold the last entry's count into rr
      r[NR - 1] = rr;
      c[NR - 1] += cc;
    } else if (can_drop) {
#pragma unroll
      for (int t = NR - 1; t > 0; --t) {
        bool sh = t > pos;
        bool here = t == pos;
        r[t] = sh ? r[t - 1] : (here ? rr : r[t]);
        c[t] = sh ? c[t - 1] : (here ? cc : c[t]);
      }
      if (pos == 0) {
        r[0] = rr;
        c[0] = cc;
      }
    } else {
      // add the count to the first entry with radius >= rr (entry `pos`)
#pragma unroll
      for (int t = 0; t < NR; ++t)
        if (t == pos) c[t] += cc;
    }
    update_rad(k);
  }
};

// ------------------------------------------------------------------ NodeToNode (kNN)
template <int NR, bool PER>
__global__ void __launch_bounds__(128) k_n2n_knn(const int32_t* __restrict__ spl_par,
                                                 const uint2* __restrict__ ilo_par,
                                                 const NodeRec* __restrict__ nodes,
                                                 uint2* __restrict__ ilo_out, IEntry* arena,
                                                 int par_plane, int k, float L, int64_t cap_ilist,
                                                 int64_t ws_total, Meta* m) {
  if (warp_failed(m)) return;
  const int64_t npar = m->n_nodes[par_plane];
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t P = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; P < npar; P += nw) {
    const int c_begin = spl_par[P], c_end = spl_par[P + 1];
    const uint2 lo = ilo_par[P];
    const uint32_t e_off = lo.x, e_cnt = lo.y & ~kUnsortedBit;
    const bool sorted = (lo.y & kUnsortedBit) == 0;
    const int C = c_end - c_begin;
    int G = 1;
    while (G < 32 && 2 * G * C <= 32) G *= 2;
    const int per = 32 / G;
    for (int c0 = c_begin; c0 < c_end; c0 += per) {
      const int cl = c0 + lane / G;
      const int sub = lane & (G - 1);
      const bool act = cl < c_end;
      NodeRec me;
      if (act) me = nodes[cl];
      else {
        me.lo[0] = me.lo[1] = me.lo[2] = 0.0f;
        me.hi[0] = me.hi[1] = me.hi[2] = 0.0f;
        me.count = 0;
        me.first = 0;
      }
      // ---- FindRmax
      RHeap<NR> H;
      H.init();
      for (uint32_t e = 0; e < e_cnt; ++e) {
        const IEntry en = arena[e_off + e];
        const bool need = act && en.r2low < H.rad;
        if (!__any_sync(kFull, need)) {
          if (sorted) break;
          continue;
        }
        const int s0 = spl_par[en.src], s1 = spl_par[en.src + 1];
        for (int jj = s0; jj < s1; jj += G) {
          const int j = jj + sub;
          if (need && j < s1) {
            const NodeRec o = nodes[j];
            const float r2 = box_dup2<PER>(me.lo, me.hi, o.lo, o.hi, L);
            if (r2 < H.rad) H.insert(r2, o.count, k);
          }
        }
      }
      for (int st = 1; st < G; st <<= 1) {
        float sr[NR];
        int sc[NR];
#pragma unroll
        for (int t = 0; t < NR; ++t) {  // snapshot: the partner reads the pre-merge heap
          sr[t] = H.r[t];
          sc[t] = H.c[t];
        }
#pragma unroll
        for (int t = 0; t < NR; ++t) {
          const float rr = __shfl_xor_sync(kFull, sr[t], st);
          const int cc = __shfl_xor_sync(kFull, sc[t], st);
          if (act && cc > 0 && rr < H.rad) H.insert(rr, cc, k);
        }
      }
      const float R2 = __shfl_sync(kFull, H.rad, lane & ~(G - 1));
      // ---- Count
      uint32_t cnt = 0;
      for (uint32_t e = 0; e < e_cnt; ++e) {
        const IEntry en = arena[e_off + e];
        const bool need = act && en.r2low <= R2;
        if (!__any_sync(kFull, need)) {
          if (sorted) break;
          continue;
        }
        const int s0 = spl_par[en.src], s1 = spl_par[en.src + 1];
        for (int j = s0 + sub; j < s1; j += G) {
          if (need) {
            const NodeRec o = nodes[j];
            cnt += box_dlow2<PER>(me.lo, me.hi, o.lo, o.hi, L) <= R2 ? 1u : 0u;
          }
        }
      }
      uint32_t tot = cnt;
      for (int st = 1; st < G; st <<= 1) tot += __shfl_xor_sync(kFull, tot, st);
      const uint32_t incl = warp_incl_scan_u(cnt);
      const uint32_t excl = incl - cnt;
      const uint32_t wtot = __shfl_sync(kFull, incl, 31);
      unsigned long long base = 0;
      if (lane == 0 && wtot) base = atomicAdd(&m->arena_used, (unsigned long long)wtot);
      base = __shfl_sync(kFull, base, 0);
      const bool ok = base + wtot <= (unsigned long long)cap_ilist;
      if (!ok) {
        if (lane == 0) {
          set_error(m, JZT_ERR_CAPACITY, kStageWalk);
          atomicMax(reinterpret_cast<unsigned long long*>(&m->required_bytes),
                    (unsigned long long)(ws_total + (int64_t)(base + wtot - cap_ilist) * (int64_t)sizeof(IEntry)));
        }
      } else {
        // ---- Insert
        unsigned long long pos = base + excl;
        for (uint32_t e = 0; e < e_cnt; ++e) {
          const IEntry en = arena[e_off + e];
          const bool need = act && en.r2low <= R2;
          if (!__any_sync(kFull, need)) {
            if (sorted) break;
            continue;
          }
          const int s0 = spl_par[en.src], s1 = spl_par[en.src + 1];
          for (int j = s0 + sub; j < s1; j += G) {
            if (need) {
              const NodeRec o = nodes[j];
              const float d2 = box_dlow2<PER>(me.lo, me.hi, o.lo, o.hi, L);
              if (d2 <= R2) {
                IEntry w;
                w.src = j;
                w.r2low = d2;
                arena[pos++] = w;
              }
            }
          }
        }
      }
      const uint32_t gexcl = __shfl_sync(kFull, excl, lane & ~(G - 1));
      if (act && sub == 0) ilo_out[cl] = ok ? make_uint2((uint32_t)(base + gexcl), tot) : make_uint2(0u, 0u);
    }
  }
}

// ------------------------------------------------------------------ list sort
// Sort one receiver's list by (r_low^2, src) with a warp bitonic network over
// 32*E register slots (lane l holds slots l*E .. l*E+E-1).  Longer lists are
// left unsorted and flagged, which disables the early exit for them.
template <int E>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&v)[E]) {
  const int lane = lane_id();
  constexpr int N = 32 * E;
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= E) {
        const int lstride = stride / E;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = lane * E + e;
          const unsigned long long o = __shfl_xor_sync(kFull, v[e], lstride);
          const bool up = (i & size) == 0;
          const bool lower = (i & stride) == 0;
          const bool keep_min = (lower == up);
          v[e] = keep_min ? (v[e] < o ? v[e] : o) : (v[e] < o ? o : v[e]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int p = e ^ stride;
          if (p > e) {
            const int i = lane * E + e;
            const bool up = (i & size) == 0;
            unsigned long long a = v[e], b = v[p];
            const bool sw = up ? (a > b) : (a < b);
            v[e] = sw ? b : a;
            v[p] = sw ? a : b;
          }
        }
      }
    }
  }
}

// Order of a receiver's list: by the squared distance between node-box centres
// (nearest first), so that the running k-th distance of a walk shrinks early;
// ties by r_low^2, then by source index.  After sorting, every entry's r_low^2 is
// replaced by the minimum r_low^2 of itself and all later entries (rounded down
// to bf16 precision: still a lower bound), so "stop once r_low^2 exceeds the
// threshold" stays exact along the list.
template <int E, bool PER>
__device__ __forceinline__ void sort_list(IEntry* list, uint32_t cnt, const NodeRec& me,
                                          const NodeRec* __restrict__ src_nodes, float L) {
  const int lane = lane_id();
  unsigned long long v[E];
  float ca[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) ca[d] = 0.5f * (me.lo[d] + me.hi[d]);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = lane * E + e;
    if (i < cnt) {
      const IEntry x = list[i];
      const NodeRec o = src_nodes[x.src];
      float c2 = 0.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float dd = 0.5f * (o.lo[d] + o.hi[d]) - ca[d];
        if (PER) dd -= L * rintf(dd / L);
        c2 = fmaf(dd, dd, c2);
      }
      const unsigned long long k16 = __float_as_uint(c2) >> 16;
      const unsigned long long r16 = __float_as_uint(x.r2low) >> 16;  // truncation rounds down
      v[e] = (k16 << 48) | (r16 << 32) | (uint32_t)x.src;
    } else {
      v[e] = ~0ull;
    }
  }
  warp_bitonic<E>(v);
  // suffix minimum of r16 (pads count as +inf)
  uint32_t r[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = lane * E + e;
    r[e] = i < cnt ? (uint32_t)((v[e] >> 32) & 0xffffu) : 0x7f80u;
  }
#pragma unroll
  for (int e = E - 2; e >= 0; --e) r[e] = min(r[e], r[e + 1]);
  uint32_t tail = r[0];  // this lane's minimum
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_down_sync(kFull, tail, o);
    if (lane + o < 32) tail = min(tail, t);
  }
  // tail now holds min over lanes >= lane; exclude this lane's own part
  uint32_t later = __shfl_down_sync(kFull, tail, 1);
  if (lane == 31) later = 0x7f80u;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = lane * E + e;
    if (i < cnt) {
      IEntry x;
      x.src = (int32_t)(uint32_t)(v[e] & 0xffffffffull);
      x.r2low = __uint_as_float(min(r[e], later) << 16);
      list[i] = x;
    }
  }
}

template <bool PER>
__global__ void __launch_bounds__(128) k_sort_lists(uint2* ilo, IEntry* arena,
                                                    const NodeRec* __restrict__ nodes, int plane,
                                                    float L, Meta* m) {
  if (warp_failed(m)) return;
  const int64_t nn = m->n_nodes[plane];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < nn; c += nw) {
    const uint2 lo = ilo[c];
    const uint32_t cnt = lo.y;
    IEntry* list = arena + lo.x;
    if (cnt <= 1) continue;
    const NodeRec me = nodes[c];
    if (cnt <= 32) sort_list<1, PER>(list, cnt, me, nodes, L);
    else if (cnt <= 64) sort_list<2, PER>(list, cnt, me, nodes, L);
    else if (cnt <= 128) sort_list<4, PER>(list, cnt, me, nodes, L);
    else if (cnt <= 256) sort_list<8, PER>(list, cnt, me, nodes, L);
    else if (lane_id() == 0) ilo[c] = make_uint2(lo.x, cnt | kUnsortedBit);
  }
}

// ------------------------------------------------------------------ LeafToLeaf (kNN)
template <int KMAX>
struct TopK {
  float d[KMAX];
  int i[KMAX];
  __device__ __forceinline__ void init(int k) {
#pragma unroll
    for (int e = 0; e < KMAX; ++e) {
      const bool pad = e < KMAX - k;  // front padding keeps the k-th entry last
      d[e] = pad ? -INFINITY : INFINITY;
      i[e] = pad ? -1 : INT_MAX;
    }
  }
  __device__ __forceinline__ float thr_d() const { return d[KMAX - 1]; }
  __device__ __forceinline__ int thr_i() const { return i[KMAX - 1]; }
  __device__ __forceinline__ bool beats(float dd, int ii) const {
    return dd < d[KMAX - 1] || (dd == d[KMAX - 1] && ii < i[KMAX - 1]);
  }
  // sorted insertion by (d, i); the last entry falls off
  __device__ __forceinline__ void insert(float dd, int ii) {
#pragma unroll
    for (int e = 0; e < KMAX; ++e) {
      const bool lt = dd < d[e] || (dd == d[e] && ii < i[e]);
      const float td = d[e];
      const int ti = i[e];
      d[e] = lt ? dd : td;
      i[e] = lt ? ii : ti;
      dd = lt ? td : dd;
      ii = lt ? ti : ii;
    }
  }
};

__device__ __forceinline__ float wrap1(float d, float L, float invL) {
  return d - L * rintf(d * invL);
}

template <bool PER>
__device__ __forceinline__ float point_box_d2(float4 q, const NodeRec& b, float L) {
  float s = 0.0f;
  const float qq[3] = {q.x, q.y, q.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float g = PER ? gap_rd_per(qq[d], qq[d], b.lo[d], b.hi[d], L)
                        : gap_rd(qq[d], qq[d], b.lo[d], b.hi[d]);
    s = __fmaf_rd(g, g, s);
  }
  return s * kLowSlack;
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
// Bounded wait on a stage barrier; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

constexpr int kQCap = 16;      // queued candidates per lane before a merge
constexpr int kL2LWarps = 4;
constexpr int kStages = 4;     // source leaves in flight per warp
constexpr int kUnroll = 4;     // source points per vote

struct __align__(16) L2LWarpSmem {
  float4 pts[kStages][32];      // staged source leaves (<= 32 points each)
  uint64_t bar[kStages];
  float qd[kQCap][32];
  int qi[kQCap][32];
};

// Per-leaf-pair distance mode (uniform over the warp): 0 plain, 1 fixed image
// shift, 2 per-pair minimum image.
template <bool PER>
__device__ __forceinline__ int pair_mode(const NodeRec& A, float bl0, float bl1, float bl2, float bh0,
                                         float bh1, float bh2, float L, float* sh) {
  if (!PER) return 0;
  const float halfL = 0.5f * L;
  const float blo[3] = {bl0, bl1, bl2}, bhi[3] = {bh0, bh1, bh2};
  bool amb = false, any = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float dlo = __fsub_rd(blo[d], A.hi[d]);
    const float dhi = __fsub_ru(bhi[d], A.lo[d]);
    sh[d] = 0.0f;
    if (dlo >= -halfL && dhi <= halfL) {
    } else if (dlo >= halfL) {
      sh[d] = -L;
      any = true;
    } else if (dhi <= -halfL) {
      sh[d] = L;
      any = true;
    } else {
      amb = true;
    }
  }
  return amb ? 2 : (any ? 1 : 0);
}

template <int MODE>
__device__ __forceinline__ float pair_d2(const float4& p, const float4& q, const float* sh, float L,
                                         float invL) {
  float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
  if (MODE == 1) {
    dx = __fadd_rn(dx, sh[0]);
    dy = __fadd_rn(dy, sh[1]);
    dz = __fadd_rn(dz, sh[2]);
  } else if (MODE == 2) {
    dx = wrap1(dx, L, invL);
    dy = wrap1(dy, L, invL);
    dz = wrap1(dz, L, invL);
  }
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Scan one staged source leaf: every (query lane, source point) pair; distances
// at or below the lane's k-th distance are queued, the queue is merged into the
// top-k when any lane's queue is nearly full.
template <int MODE, int KMAX>
__device__ __forceinline__ void scan_leaf(const float4* __restrict__ sp, int cnt, int G, int sub,
                                          const float4& qp, const float* sh, float L, float invL,
                                          TopK<KMAX>& T, float& thr, int& qn, float (*qd)[32],
                                          int (*qi)[32], int lane, bool act) {
  for (int j0 = 0; j0 < cnt; j0 += kUnroll * G) {
    float d2[kUnroll];
    int id[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int j = j0 + u * G + sub;  // slots past cnt hold +inf points
      const float4 p = sp[j < 32 ? j : 31];
      d2[u] = pair_d2<MODE>(p, qp, sh, L, invL);
      id[u] = __float_as_int(p.w);
      if (j >= 32) d2[u] = INFINITY;
    }
    bool c = false;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) c |= d2[u] <= thr;
    if (__any_sync(kFull, c)) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (d2[u] <= thr) {
          qd[qn][lane] = d2[u];
          qi[qn][lane] = id[u];
          ++qn;
        }
      }
      if (__any_sync(kFull, qn > kQCap - kUnroll)) {
        for (int t = 0; t < qn; ++t) {
          const float dd = qd[t][lane];
          const int ii = qi[t][lane];
          if (T.beats(dd, ii)) T.insert(dd, ii);
        }
        qn = 0;
        thr = act ? T.thr_d() : -INFINITY;
      }
    }
  }
}

// One warp per query leaf.  Source leaves of the (sorted) interaction list are
// staged into shared memory by bulk copies, kStages ahead of the computation;
// the list metadata (source box and point range) is read 32 entries at a time,
// one entry per lane.
template <int KMAX, bool PER>
__global__ void __launch_bounds__(32 * kL2LWarps) k_l2l_knn(const float4* __restrict__ pts,
                                                           const NodeRec* __restrict__ leaves,
                                                           const uint2* __restrict__ ilo,
                                                           const IEntry* __restrict__ arena, int k,
                                                           float L, int order,
                                                           int32_t* __restrict__ out_idx,
                                                           float* __restrict__ out_d2, Meta* m) {
  __shared__ L2LWarpSmem S_all[kL2LWarps];
  if (warp_failed(m)) return;
  const int w = warp_id(), lane = lane_id();
  L2LWarpSmem& S = S_all[w];
  if (lane == 0) {
    for (int t = 0; t < kStages; ++t) mbar_init(&S.bar[t], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  uint32_t parity = 0;  // bit t: parity of the next completion of stage t
  const int64_t nl = m->n_nodes[0];
  const float invL = PER ? 1.0f / L : 0.0f;
  bool broken = false;
  while (!broken) {
    int64_t leaf = 0;
    if (lane == 0) leaf = atomicAdd(&m->tile_ctr[kCtrWalk], 1u);
    leaf = __shfl_sync(kFull, leaf, 0);
    if (leaf >= nl) break;
    const NodeRec me = leaves[leaf];
    const int q = me.count;
    int G = 1;
    while (G < 32 && 2 * G * q <= 32) G *= 2;
    const int qi = lane / G, sub = lane & (G - 1);
    const bool act = qi < q;
    const float4 qp = act ? pts[me.first + qi] : make_float4(0.f, 0.f, 0.f, 0.f);
    TopK<KMAX> T;
    T.init(k);
    float thr = act ? T.thr_d() : -INFINITY;
    int qn = 0;
    unsigned long long pairs = 0;
    const uint2 lo = ilo[leaf];
    const uint32_t e_cnt = lo.y & ~kUnsortedBit;
    const bool sorted = (lo.y & kUnsortedBit) == 0;
    const IEntry* list = arena + lo.x;
    bool stop = false;  // sorted list and every later entry beyond all thresholds

    for (uint32_t b0 = 0; b0 < e_cnt && !broken && !stop; b0 += 32) {
      const uint32_t nb = min(32u, e_cnt - b0);
      // metadata of up to 32 entries, one per lane
      IEntry en;
      en.src = 0;
      en.r2low = INFINITY;
      NodeRec sr;
      if ((uint32_t)lane < nb) {
        en = list[b0 + lane];
        sr = leaves[en.src];
      } else {
        sr.count = 0;
        sr.first = 0;
      }
      uint32_t issued = 0, done = 0;
      auto issue = [&](uint32_t e) {
        const float r2 = __shfl_sync(kFull, en.r2low, e);
        const bool reach = act && r2 <= thr;
        if (sorted && !__any_sync(kFull, reach)) {
          stop = true;
          return;
        }
        const int first = __shfl_sync(kFull, sr.first, e);
        const int cnt = __shfl_sync(kFull, sr.count, e);
        const int st = e % kStages;
        __syncwarp();
        if (lane == 0) {
          fence_proxy_async();
          mbar_expect_tx(&S.bar[st], (uint32_t)cnt * 16u);
          bulk_g2s(&S.pts[st][0], pts + first, (uint32_t)cnt * 16u, &S.bar[st]);
        }
        ++issued;
      };
      while (issued < nb && issued < (uint32_t)kStages && !stop) issue(issued);
      while (done < issued) {
        const uint32_t e = done;
        const int st = e % kStages;
        const bool landed = __all_sync(kFull, mbar_wait(&S.bar[st], (parity >> st) & 1u));
        if (!landed) {
          if (lane == 0) set_error(m, JZT_ERR_TIMEOUT, kStageLeaf);
          broken = true;
          // give the copies still in flight a bounded chance to land before leaving
          for (uint32_t r = done + 1; r < issued; ++r) {
            const int s2 = r % kStages;
            (void)__all_sync(kFull, mbar_wait(&S.bar[s2], (parity >> s2) & 1u));
          }
          break;
        }
        parity ^= 1u << st;
        ++done;
        const int cnt = __shfl_sync(kFull, sr.count, e);
        // pad the stage with far-away points so the unrolled scan needs no bounds
        if (lane >= cnt) S.pts[st][lane] = make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(INT_MAX));
        __syncwarp();
        const float r2 = __shfl_sync(kFull, en.r2low, e);
        const bool reach = act && r2 <= thr;
        bool skip = !__any_sync(kFull, reach);
        if (skip && sorted) stop = true;
        float bl[3], bh[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          bl[d] = __shfl_sync(kFull, sr.lo[d], e);
          bh[d] = __shfl_sync(kFull, sr.hi[d], e);
        }
        if (!skip) {
          // point-to-box lower bound against this lane's threshold
          float pb = 0.0f;
          const float qq[3] = {qp.x, qp.y, qp.z};
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float g = PER ? gap_rd_per(qq[d], qq[d], bl[d], bh[d], L) : gap_rd(qq[d], qq[d], bl[d], bh[d]);
            pb = __fmaf_rd(g, g, pb);
          }
          skip = !__any_sync(kFull, act && pb * kLowSlack <= thr);
        }
        if (!skip) {
          pairs += (unsigned long long)q * (unsigned long long)cnt;
          float sh[3];
          const int mode = pair_mode<PER>(me, bl[0], bl[1], bl[2], bh[0], bh[1], bh[2], L, sh);
          if (mode == 0) scan_leaf<0, KMAX>(S.pts[st], cnt, G, sub, qp, sh, L, invL, T, thr, qn, S.qd, S.qi, lane, act);
          else if (mode == 1) scan_leaf<1, KMAX>(S.pts[st], cnt, G, sub, qp, sh, L, invL, T, thr, qn, S.qd, S.qi, lane, act);
          else scan_leaf<2, KMAX>(S.pts[st], cnt, G, sub, qp, sh, L, invL, T, thr, qn, S.qd, S.qi, lane, act);
        }
        __syncwarp();
        if (!stop && issued < nb) issue(issued);
      }
    }
    // merge what is still queued
    for (int t = 0; t < qn; ++t) {
      const float dd = S.qd[t][lane];
      const int ii = S.qi[t][lane];
      if (T.beats(dd, ii)) T.insert(dd, ii);
    }
    __syncwarp();
    // merge the G partial lists of each query (butterfly; lists stay exact)
    for (int st = 1; st < G; st <<= 1) {
      TopK<KMAX> snap = T;  // the partner reads the pre-merge list
#pragma unroll
      for (int e = 0; e < KMAX; ++e) {
        const float dd = __shfl_xor_sync(kFull, snap.d[e], st);
        const int ii = __shfl_xor_sync(kFull, snap.i[e], st);
        if (act && dd >= 0.0f && T.beats(dd, ii)) T.insert(dd, ii);
      }
    }
    if (lane == 0 && pairs) atomicAdd(&m->knn_pairs, pairs);
    if (act && sub == 0 && !broken) {
      const int64_t row = order == 0 ? (int64_t)__float_as_int(qp.w) : (int64_t)(me.first + qi);
      int32_t* oi = out_idx + row * k;
      float* od = out_d2 + row * k;
#pragma unroll
      for (int e = 0; e < KMAX; ++e) {
        if (e >= KMAX - k) {
          oi[e - (KMAX - k)] = T.i[e];
          od[e - (KMAX - k)] = T.d[e];
        }
      }
    }
    __syncwarp();
  }
}

__global__ void k_walk_peak(Meta* m) {
  if (threadIdx.x == 0) m->arena_peak = m->arena_used;
}

int grid_for(int64_t work, int threads, int max_blocks) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

template <int NR, bool PER>
void n2n_knn_plane(const Layout& L, char* ws, int p, int k, float pl, cudaStream_t s) {
  Meta* m = at<Meta>(ws, L.meta);
  const int sms = 152;
  k_n2n_knn<NR, PER><<<grid_for(L.cap_nodes[p + 1] * 32, 128, sms * 16), 128, 0, s>>>(
      at<int32_t>(ws, L.spl[p + 1]), at<uint2>(ws, L.ilo[p + 1]), at<NodeRec>(ws, L.nodes[p]),
      at<uint2>(ws, L.ilo[p]), at<IEntry>(ws, L.arena), p + 1, k, pl, L.cap_ilist,
      (int64_t)L.total, m); note_launch();
}

template <int KMAX, bool PER>
void l2l_knn(const Layout& L, char* ws, int k, float pl, int order, int32_t* idx, float* d2,
             cudaStream_t s) {
  Meta* m = at<Meta>(ws, L.meta);
  const int sms = 152;
  k_l2l_knn<KMAX, PER><<<sms * 8, 32 * kL2LWarps, 0, s>>>(
      at<float4>(ws, L.pts), at<NodeRec>(ws, L.nodes[0]), at<uint2>(ws, L.ilo[0]),
      at<IEntry>(ws, L.arena), k, pl, order, idx, d2, m); note_launch();
}

template <bool PER>
void knn_all(const Layout& L, char* ws, float pl, int k, int order, int32_t* idx, float* d2,
             cudaStream_t s) {
  Meta* m = at<Meta>(ws, L.meta);
  const int sms = 152;
  const int P = L.n_planes;
  prof_begin(kPhKnnTop, s);
  k_walk_reset<<<1, 32, 0, s>>>(m); note_launch();
  launch_super_level(L, ws, s);
  k_dense_ilist<<<grid_for(L.cap_nodes[P], 128, sms * 4), 128, 0, s>>>(
      m, at<uint2>(ws, L.ilo[P]), at<IEntry>(ws, L.arena), P, 0, L.cap_ilist, m); note_launch();
  prof_end(kPhKnnTop, s);
  for (int p = P - 1; p >= 0; --p) {
    prof_begin(kPhKnnN2N, s);
    if (L.heap <= 4) n2n_knn_plane<4, PER>(L, ws, p, k, pl, s);
    else if (L.heap <= 8) n2n_knn_plane<8, PER>(L, ws, p, k, pl, s);
    else n2n_knn_plane<16, PER>(L, ws, p, k, pl, s);
    prof_end(kPhKnnN2N, s);
    prof_begin(kPhKnnSort, s);
    k_sort_lists<PER><<<grid_for(L.cap_nodes[p] * 32, 128, sms * 16), 128, 0, s>>>(
        at<uint2>(ws, L.ilo[p]), at<IEntry>(ws, L.arena), at<NodeRec>(ws, L.nodes[p]), p, pl, m); note_launch();
    prof_end(kPhKnnSort, s);
  }
  prof_begin(kPhKnnL2L, s);
  if (k <= 4) l2l_knn<4, PER>(L, ws, k, pl, order, idx, d2, s);
  else if (k <= 8) l2l_knn<8, PER>(L, ws, k, pl, order, idx, d2, s);
  else if (k <= 16) l2l_knn<16, PER>(L, ws, k, pl, order, idx, d2, s);
  else l2l_knn<32, PER>(L, ws, k, pl, order, idx, d2, s);
  prof_end(kPhKnnL2L, s);
  k_walk_peak<<<1, 32, 0, s>>>(m); note_launch();
}

}  // namespace

void launch_knn(const Layout& L, char* ws, float periodic_L, int k, int order, int32_t* d_idx,
                float* d_d2, cudaStream_t s) {
  if (periodic_L > 0.0f) knn_all<true>(L, ws, periodic_L, k, order, d_idx, d_d2, s);
  else knn_all<false>(L, ws, 0.0f, k, order, d_idx, d_d2, s);
}

}  // namespace jzt
