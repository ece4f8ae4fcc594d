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
#include <cstring>

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
  if (threadIdx.x < 8) m->knn_stats[threadIdx.x] = 0;
  if (threadIdx.x < kMaxPlanes) m->knn_plane_entries[threadIdx.x] = 0;
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
constexpr int kN2NWarps = 4;
constexpr int kMetaCap = 256;  // list entries whose metadata a warp caches in shared memory

struct __align__(16) N2NWarpSmem {
  float ent_r2[kMetaCap];   // r_low^2 of each list entry
  int ent_s0[kMetaCap];     // first child (global index) of the entry's source
  int ent_cnt[kMetaCap];    // children of the entry's source
  int ent_code[kMetaCap];   // image code of the source relative to the receiver (periodic)
};

// Image code of a source box relative to a receiver box in a periodic box:
// bits 0-5 hold, per dimension, 0 (no shift), 1 (+L) or 2 (-L) when that image is
// the minimum image for every pair of points of the two boxes; bit 6 = ambiguous.
template <bool PER>
__device__ __forceinline__ int image_code(const float* alo, const float* ahi, const float* blo,
                                          const float* bhi, float L) {
  if (!PER) return 0;
  const float halfL = 0.5f * L;
  int code = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float dlo = __fsub_rd(blo[d], ahi[d]);
    const float dhi = __fsub_ru(bhi[d], alo[d]);
    if (dlo >= -halfL && dhi <= halfL) {
    } else if (dhi <= -halfL) {
      code |= 1 << (2 * d);
    } else if (dlo >= halfL) {
      code |= 2 << (2 * d);
    } else {
      code |= 64;
    }
  }
  return code;
}

// Box-box bounds with a fixed image: the source box is shifted by the code's
// image (rounded outward) and the open-box formulas apply; ambiguous pairs use
// the minimum over the images.
template <bool PER, bool UP>
__device__ __forceinline__ float box_bound2(const NodeRec& a, const NodeRec& b, int code, float L) {
  if (PER && (code & 64)) {
    return UP ? box_dup2<true>(a.lo, a.hi, b.lo, b.hi, L) : box_dlow2<true>(a.lo, a.hi, b.lo, b.hi, L);
  }
  float blo[3], bhi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int c = PER ? (code >> (2 * d)) & 3 : 0;
    const float sh = c == 1 ? L : (c == 2 ? -L : 0.0f);
    blo[d] = c ? __fadd_rd(b.lo[d], sh) : b.lo[d];
    bhi[d] = c ? __fadd_ru(b.hi[d], sh) : b.hi[d];
  }
  return UP ? box_dup2<false>(a.lo, a.hi, blo, bhi, L) : box_dlow2<false>(a.lo, a.hi, blo, bhi, L);
}

// Squared distance between box centres under the code's image (ordering only).
template <bool PER>
__device__ __forceinline__ float centre_d2(const NodeRec& a, const NodeRec& b, int code, float L) {
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float dd = 0.5f * (b.lo[d] + b.hi[d]) - 0.5f * (a.lo[d] + a.hi[d]);
    if (PER) {
      if (code & 64) dd -= L * rintf(dd / L);
      else {
        const int c = (code >> (2 * d)) & 3;
        dd += c == 1 ? L : (c == 2 ? -L : 0.0f);
      }
    }
    s = fmaf(dd, dd, s);
  }
  return s;
}

// Internal radius bound of every node of plane p >= 1, bottom-up: for each child
// c, the smallest radius whose d_up-ball holds k points of its siblings (itself
// included; RadiusOfCount over the parent's own children, Alg. 3's heap) and,
// when c has children, c's own bound; the node's bound is the largest over its
// children.  Every point of the node has its k nearest neighbours within it, so
// it caps the node's R_max in the walk.  One warp per node.
template <int NR, bool PER>
__global__ void __launch_bounds__(128) k_internal_bounds(const int32_t* __restrict__ spl,
                                                         const NodeRec* __restrict__ child,
                                                         const float* __restrict__ rint_child,
                                                         float* __restrict__ rint, int plane, int k,
                                                         float L, const Meta* m) {
  if (warp_failed(m)) return;
  const int64_t nn = m->n_nodes[plane];
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t P = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; P < nn; P += nw) {
    const int s0 = spl[P], s1 = spl[P + 1];
    float worst = 0.0f;
    for (int c0 = s0; c0 < s1; c0 += 32) {
      const int c = c0 + lane;
      const bool act = c < s1;
      NodeRec me;
      if (act) me = child[c];
      else {
        me.lo[0] = me.lo[1] = me.lo[2] = 0.0f;
        me.hi[0] = me.hi[1] = me.hi[2] = 0.0f;
      }
      const float own = (act && rint_child != nullptr) ? rint_child[c] : INFINITY;
      RHeap<NR> H;
      H.init();
      for (int sb = s0; sb < s1; ++sb) {
        const NodeRec o = child[sb];
        const float u2 = box_dup2<PER>(me.lo, me.hi, o.lo, o.hi, L);
        if (act && u2 < fminf(H.rad, own)) H.insert(u2, o.count, k);
      }
      if (act) worst = fmaxf(worst, fminf(H.rad, own));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(kFull, worst, o));
    if (lane == 0) rint[P] = worst;
  }
}

// One warp per receiving parent; G lanes per child split the candidates (the
// children of the parent's source parents).  The list metadata (first child,
// child count, r_low^2 and image code of each source) is gathered once per
// parent, 32 entries at a time, into shared memory.
template <int NR, bool PER>
__global__ void __launch_bounds__(32 * kN2NWarps) k_n2n_knn(const int32_t* __restrict__ spl_par,
                                                            const uint2* __restrict__ ilo_par,
                                                            const NodeRec* __restrict__ par_nodes,
                                                            const NodeRec* __restrict__ nodes,
                                                            const float* __restrict__ rint,
                                                            uint2* __restrict__ ilo_out, IEntry* arena,
                                                            int par_plane, int k, float L,
                                                            int64_t cap_ilist, int64_t ws_total,
                                                            Meta* m) {
  __shared__ N2NWarpSmem S_all[kN2NWarps];
  if (warp_failed(m)) return;
  const int lane = lane_id();
  N2NWarpSmem& S = S_all[warp_id()];
  const int64_t npar = m->n_nodes[par_plane];
  // parents are taken one at a time from a shared counter (their cost varies with
  // their children and lists; a fixed stride left warps idle at the end)
  while (true) {
    int64_t P = 0;
    if (lane == 0) P = atomicAdd(&m->tile_ctr[kCtrN2N], 1u);
    P = __shfl_sync(kFull, P, 0);
    if (P >= npar) break;
    const int c_begin = spl_par[P], c_end = spl_par[P + 1];
    const uint2 lo = ilo_par[P];
    const uint32_t e_off = lo.x, e_cnt = lo.y & ~kUnsortedBit;
    const bool sorted = (lo.y & kUnsortedBit) == 0;
    // receiver box for image codes; the super level has no records (codes = ambiguous)
    NodeRec pb;
    const bool have_par = par_nodes != nullptr;
    if (have_par) pb = par_nodes[P];
    auto load_meta = [&](uint32_t e, float& r2, int& s0, int& cnt, int& code) {
      IEntry en = arena[e_off + e];
      if ((uint64_t)(uint32_t)en.src >= (uint64_t)npar) {  // consistency guard
        set_error(m, JZT_ERR_INTERNAL, kStageWalk);
        en.src = 0;
        en.r2low = INFINITY;
      }
      r2 = en.r2low;
      s0 = spl_par[en.src];
      cnt = spl_par[en.src + 1] - s0;
      if (PER) {
        if (have_par) {
          const NodeRec sb = par_nodes[en.src];
          code = image_code<PER>(pb.lo, pb.hi, sb.lo, sb.hi, L);
        } else {
          code = 64;
        }
      } else {
        code = 0;
      }
    };
    const uint32_t n_cached = min(e_cnt, (uint32_t)kMetaCap);
    for (uint32_t e = lane; e < n_cached; e += 32) {
      float r2;
      int s0, cnt, code;
      load_meta(e, r2, s0, cnt, code);
      S.ent_r2[e] = r2;
      S.ent_s0[e] = s0;
      S.ent_cnt[e] = cnt;
      S.ent_code[e] = code;
    }
    __syncwarp();
    auto entry = [&](uint32_t e, float& r2, int& s0, int& cnt, int& code) {
      if (e < (uint32_t)kMetaCap) {
        r2 = S.ent_r2[e];
        s0 = S.ent_s0[e];
        cnt = S.ent_cnt[e];
        code = S.ent_code[e];
      } else {
        load_meta(e, r2, s0, cnt, code);
      }
    };

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
      // ---- FindRmax (Alg. 3), capped by the node's internal bound (no candidate
      // at or beyond the cap can lower the result below it)
      const float cap2 = (rint != nullptr && act) ? rint[cl] : INFINITY;
      RHeap<NR> H;
      H.init();
      for (uint32_t e = 0; e < e_cnt; ++e) {
        float r2;
        int s0, cnt, code;
        entry(e, r2, s0, cnt, code);
        const bool need = act && r2 < fminf(H.rad, cap2);
        if (!__any_sync(kFull, need)) {
          if (sorted) break;
          continue;
        }
        for (int j = sub; j < cnt; j += G) {
          if (need) {
            const NodeRec o = nodes[s0 + j];
            const float u2 = box_bound2<PER, true>(me, o, code, L);
            if (u2 < fminf(H.rad, cap2)) H.insert(u2, o.count, k);
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
      const float R2 = fminf(__shfl_sync(kFull, H.rad, lane & ~(G - 1)), cap2);
      // ---- Count
      uint32_t cnt_out = 0;
      for (uint32_t e = 0; e < e_cnt; ++e) {
        float r2;
        int s0, cnt, code;
        entry(e, r2, s0, cnt, code);
        const bool need = act && r2 <= R2;
        if (!__any_sync(kFull, need)) {
          if (sorted) break;
          continue;
        }
        for (int j = sub; j < cnt; j += G) {
          if (need) cnt_out += box_bound2<PER, false>(me, nodes[s0 + j], code, L) <= R2 ? 1u : 0u;
        }
      }
      uint32_t tot = cnt_out;
      for (int st = 1; st < G; st <<= 1) tot += __shfl_xor_sync(kFull, tot, st);
      const uint32_t incl = warp_incl_scan_u(cnt_out);
      const uint32_t excl = incl - cnt_out;
      const uint32_t wtot = __shfl_sync(kFull, incl, 31);
      unsigned long long base_out = 0;
      if (lane == 0 && wtot) base_out = atomicAdd(&m->arena_used, (unsigned long long)wtot);
      base_out = __shfl_sync(kFull, base_out, 0);
      const bool ok = base_out + wtot <= (unsigned long long)cap_ilist;
      if (!ok) {
        if (lane == 0) {
          set_error(m, JZT_ERR_CAPACITY, kStageWalk);
          atomicMax(reinterpret_cast<unsigned long long*>(&m->required_bytes),
                    (unsigned long long)(ws_total + (int64_t)(base_out + wtot - cap_ilist) * (int64_t)sizeof(IEntry)));
        }
      } else {
        // ---- Insert
        unsigned long long pos = base_out + excl;
        for (uint32_t e = 0; e < e_cnt; ++e) {
          float r2;
          int s0, cnt, code;
          entry(e, r2, s0, cnt, code);
          const bool need = act && r2 <= R2;
          if (!__any_sync(kFull, need)) {
            if (sorted) break;
            continue;
          }
          for (int j = sub; j < cnt; j += G) {
            if (need) {
              const NodeRec o = nodes[s0 + j];
              const float d2 = box_bound2<PER, false>(me, o, code, L);
              if (d2 <= R2) {
                // packed for the list sort: bf16 of the centre distance^2 (high half)
                // and of r_low^2 rounded down (low half)
                const float c2 = centre_d2<PER>(me, o, code, L);
                IEntry wr;
                wr.src = s0 + j;
                wr.r2low = __uint_as_float((__float_as_uint(c2) & 0xffff0000u) | (__float_as_uint(d2) >> 16));
                arena[pos++] = wr;
              }
            }
          }
        }
      }
      const uint32_t gexcl = __shfl_sync(kFull, excl, lane & ~(G - 1));
      if (act && sub == 0) ilo_out[cl] = ok ? make_uint2((uint32_t)(base_out + gexcl), tot) : make_uint2(0u, 0u);
    }
    __syncwarp();  // cached metadata is rewritten for the next parent
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
// ties by r_low^2, then by source index.  The NodeToNode insert stored both keys
// as bf16 halves of the r2low field.  After sorting, every entry's r_low^2 is
// replaced by the minimum r_low^2 of itself and all later entries (bf16, rounded
// down: still a lower bound), so "stop once r_low^2 exceeds the threshold" stays
// exact along the list.  Lists too long to sort in registers are only unpacked
// and flagged unsorted.
template <int E>
__device__ __forceinline__ void sort_list(IEntry* list, uint32_t cnt) {
  const int lane = lane_id();
  unsigned long long v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = lane * E + e;
    if (i < cnt) {
      const IEntry x = list[i];
      v[e] = ((unsigned long long)__float_as_uint(x.r2low) << 32) | (uint32_t)x.src;
    } else {
      v[e] = ~0ull;
    }
  }
  warp_bitonic<E>(v);
  // suffix minimum of the r_low^2 half (pads count as +inf)
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
  // tail holds the minimum over lanes >= lane; take the part after this lane
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

// Lists of 129..256 entries: the same order by a bitonic network in shared
// memory (the warp's 256 slots), so that the register-resident sorts above stay
// small and the kernel keeps many warps per SM.
__device__ __noinline__ void sort_list_smem(IEntry* list, uint32_t cnt, unsigned long long* buf) {
  const int lane = lane_id();
  for (uint32_t i = lane; i < 256; i += 32) {
    if (i < cnt) {
      const IEntry x = list[i];
      buf[i] = ((unsigned long long)__float_as_uint(x.r2low) << 32) | (uint32_t)x.src;
    } else {
      buf[i] = ~0ull;
    }
  }
  __syncwarp();
  for (int size = 2; size <= 256; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = lane; q < 128; q += 32) {  // pair q: lower index i, partner i + stride
        const int i = ((q / stride) * 2 * stride) + (q % stride);
        const int j = i + stride;
        const bool up = (i & size) == 0;
        const unsigned long long a = buf[i], b = buf[j];
        if ((a > b) == up) {
          buf[i] = b;
          buf[j] = a;
        }
      }
      __syncwarp();
    }
  }
  // r_low^2 halves made suffix minima (bf16, rounded down), written back unpacked
  uint32_t later = 0x7f80u;
  for (int c = 7; c >= 0; --c) {  // chunks of 32 from the end
    const uint32_t i = 32u * c + lane;
    uint32_t r = i < cnt ? (uint32_t)((buf[i] >> 32) & 0xffffu) : 0x7f80u;
    // suffix minimum within the chunk (lanes >= lane), then with the later chunks
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_down_sync(kFull, r, o);
      if (lane + o < 32) r = min(r, t);
    }
    r = min(r, later);
    later = __shfl_sync(kFull, r, 0);
    if (i < cnt) {
      IEntry x;
      x.src = (int32_t)(uint32_t)(buf[i] & 0xffffffffull);
      x.r2low = __uint_as_float(r << 16);
      list[i] = x;
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(128) k_sort_lists(uint2* ilo, IEntry* arena, int plane, Meta* m) {
  __shared__ unsigned long long s_buf[4][256];
  if (warp_failed(m)) return;
  const int64_t nn = m->n_nodes[plane];
  // lists are taken one at a time from a device counter (their lengths vary)
  while (true) {
    int64_t c = 0;
    if (lane_id() == 0) c = atomicAdd(&m->tile_ctr[kCtrLists], 1u);
    c = __shfl_sync(kFull, c, 0);
    if (c >= nn) break;
    const uint2 lo = ilo[c];
    const uint32_t cnt = lo.y;
    IEntry* list = arena + lo.x;
    if (cnt <= 32) sort_list<1>(list, cnt);
    else if (cnt <= 64) sort_list<2>(list, cnt);
    else if (cnt <= 128) sort_list<4>(list, cnt);
    else if (cnt <= 256) sort_list_smem(list, cnt, s_buf[warp_id()]);
    else {
      for (uint32_t i = lane_id(); i < cnt; i += 32) {
        IEntry x = list[i];
        x.r2low = __uint_as_float(__float_as_uint(x.r2low) << 16);
        list[i] = x;
      }
      if (lane_id() == 0) ilo[c] = make_uint2(lo.x, cnt | kUnsortedBit);
    }
  }
}

// ------------------------------------------------------------------ LeafToLeaf (kNN)
__device__ __forceinline__ float wrap1(float d, float L, float invL) {
  return d - L * rintf(d * invL);
}

#ifndef JZT_L2L_STAGES
#define JZT_L2L_STAGES 2
#endif
#ifndef JZT_L2L_MINBLOCKS
// blocks per SM: 5 caps registers at 96 (a few spilled words, faster than 4
// blocks without spills), 3 at 168; shared memory allows 5 blocks at
// KMAX <= 16 (two staged leaves per warp) and 3 at KMAX = 32
#define JZT_L2L_MINBLOCKS(kmax) ((kmax) <= 16 ? 5 : 3)
#endif
// Threshold updates: once a lane holds kMergeAt unmerged candidates, its oldest
// kMergeBatch are merged into the distance list.  Batches of 8 halve the sorting
// network at KMAX <= 16; at KMAX = 32 the list's own merge network dominates and
// batches of 16, merged as soon as 9 are waiting, are faster.
template <int KMAX> constexpr int kMergeBatch = KMAX <= 16 ? 8 : 16;
template <int KMAX> constexpr int kMergeAt = KMAX <= 16 ? 8 : 9;
constexpr int kL2LWarps = 4;
constexpr int kStages = JZT_L2L_STAGES;  // source leaves in flight per warp

// Exact keys are packed as (float32 bits of d2) << 32 | (original index + 1):
// for d2 >= 0 the unsigned order of the key is the order by (d2, index);
// kKeyInf, above every real key, pads the sorting networks.
constexpr unsigned long long kKeyInf = ~0ull;

// Per-warp shared memory: staged source leaves and, per lane, a buffer of
// candidate (d2 bits, original index) pairs.  The buffer holds KMAX + 16
// entries: a compaction leaves at most KMAX, and the scan compacts as soon as
// more than kCap - 8 are held after a window of 8 source points, so the next
// window always fits.
template <int KMAX>
struct __align__(16) L2LWarpSmem {
  static constexpr int kCap = KMAX + 16;
  float4 pts[kStages][32];  // staged source leaves (<= 32 points each)
  float4 meta[32][3];       // list entries of the current batch (see k_l2l_knn)
  uint64_t bar[kStages];
  uint2 buf[kCap][32];      // buf[slot][lane]
};

__device__ __forceinline__ void cswap(unsigned long long& a, unsigned long long& b) {
  const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
  a = lo;
  b = hi;
}
__device__ __forceinline__ void cswap(float& a, float& b) {
  const float lo = fminf(a, b), hi = fmaxf(a, b);
  a = lo;
  b = hi;
}

// Sorted top-K list in registers (ascending; the first K-k slots hold pads
// below every real entry so that the k-th best entry is always the last one).
// New entries are merged in batches: the batch is sorted with a bitonic
// network, paired against the list in reverse (which leaves a bitonic sequence
// holding the K smallest of both), and a bitonic merge restores the order.
// Branch-free, so lanes with different numbers of new entries do not diverge.
// T is unsigned long long for packed (d2, index) keys, float for distances only.
template <typename T, int K>
struct RegTopK {
  T t[K];
  __device__ __forceinline__ void init(int k, T pad, T inf) {
#pragma unroll
    for (int e = 0; e < K; ++e) t[e] = e < K - k ? pad : inf;
  }
  template <int B>
  __device__ __forceinline__ void merge(T (&b)[B]) {
#pragma unroll
    for (int size = 2; size <= B; size <<= 1)
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
        for (int i = 0; i < B; ++i) {
          const int j = i ^ stride;
          if (j > i) {
            if ((i & size) == 0) cswap(b[i], b[j]);
            else cswap(b[j], b[i]);
          }
        }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int j = K - 1 - i;
      if (j < B) t[i] = t[i] < b[j] ? t[i] : b[j];
    }
#pragma unroll
    for (int stride = K >> 1; stride > 0; stride >>= 1)
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int j = i ^ stride;
        if (j > i) cswap(t[i], t[j]);
      }
  }
};

// Per-lane candidate state of one query: the buffer (in shared memory) holds
// nb entries, of which the first nm have been merged into F, the k smallest
// distances seen so far; F's last entry is the running k-th distance thr.
// Every source point at or below thr when it is scanned is buffered, so the
// buffer always holds every point that can still be among the k nearest.
template <int KMAX>
struct Cand {
  RegTopK<float, KMAX> F;
  int nb, nm;
  float thr;
  uint32_t pushed;
};

// Merge the oldest unmerged buffer entries (at most kMergeBatch) into F and
// update thr.
template <int KMAX>
__device__ __forceinline__ void merge_distances(uint2 (*buf)[32], Cand<KMAX>& C, int lane, bool act) {
  constexpr int kCap = L2LWarpSmem<KMAX>::kCap;
  constexpr int B = kMergeBatch<KMAX>;
  const int take = min(B, C.nb - C.nm);
  float b[B];
#pragma unroll
  for (int t = 0; t < B; ++t) {
    const int r = t < take ? C.nm + t : 0;  // index stays inside the lane's buffer
    const float v = __uint_as_float(buf[r < kCap ? r : 0][lane].x);
    b[t] = t < take ? v : INFINITY;
  }
  C.pushed += (uint32_t)take;
  C.nm += take;
  C.F.template merge<B>(b);
  C.thr = act ? C.F.t[KMAX - 1] : -INFINITY;
}

// Descending bitonic sort of N keys in registers (N a power of two).
template <int N>
__device__ __forceinline__ void sort_desc(unsigned long long (&v)[N]) {
#pragma unroll
  for (int size = 2; size <= N; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int j = i ^ stride;
        if (j > i) {
          if ((i & size) == 0) cswap(v[j], v[i]);  // this block descending: the larger first
          else cswap(v[i], v[j]);
        }
      }
}

// Keep only the buffer entries at or below thr.  If a lane still holds more
// than KMAX (exact ties at the k-th distance), every lane also drops the tied
// entries beyond its k best: fewer than k entries lie below thr, and of those
// at thr the ones with the smallest indices are kept (indices are distinct).
template <int KMAX>
__device__ __forceinline__ void compact(uint2 (*buf)[32], Cand<KMAX>& C, int k, int lane) {
  int w = 0;
  for (int r = 0; r < C.nb; ++r) {
    const uint2 e = buf[r][lane];
    if (__uint_as_float(e.x) <= C.thr) buf[w++][lane] = e;
  }
  C.nb = C.nm = w;
  if (!__any_sync(kFull, C.nb > KMAX)) return;
  const uint32_t tb = __float_as_uint(C.thr);
  int less = 0;
  for (int r = 0; r < C.nb; ++r) less += __uint_as_float(buf[r][lane].x) < C.thr ? 1 : 0;
  uint32_t cut = 0;
  bool have = false;
  for (int t = less; t < k; ++t) {  // the (k - less)-th smallest index among the ties
    uint32_t mn = 0xffffffffu;
    for (int r = 0; r < C.nb; ++r) {
      const uint2 e = buf[r][lane];
      if (e.x == tb && (!have || e.y > cut) && e.y < mn) mn = e.y;
    }
    cut = mn;
    have = true;
  }
  w = 0;
  for (int r = 0; r < C.nb; ++r) {
    const uint2 e = buf[r][lane];
    if (__uint_as_float(e.x) < C.thr || (have && e.x == tb && e.y <= cut)) buf[w++][lane] = e;
  }
  C.nb = C.nm = w;
}

// Per-leaf-pair distance mode (uniform over the warp): 0 plain, 1 fixed image
// shift, 2 per-pair minimum image.
template <bool PER>
__device__ __forceinline__ int pair_mode(const NodeRec& A, const float* blo, const float* bhi,
                                         float L, float* sh) {
  if (!PER) return 0;
  const float halfL = 0.5f * L;
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

// Distances from the lane's query to W staged source points: slot j0 + u*G + sub
// (sub-lane sub of G lanes per query).  Slots past cnt read as NaN.
template <int MODE, int W>
__device__ __forceinline__ void window_d2(const float4* __restrict__ sp, int j0, int cnt, int G, int sub,
                                          const float4& qp, const float* sh, float L, float invL,
                                          float (&d2)[W], int (&id)[W]) {
  if (G == 1) {  // j0 + u <= 31; the staged slots past cnt already hold NaN points
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const float4 p = sp[j0 + u];
      d2[u] = pair_d2<MODE>(p, qp, sh, L, invL);
      id[u] = __float_as_int(p.w);
    }
  } else {
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const int j = j0 + u * G + sub;
      const float4 p = sp[j < 32 ? j : 31];
      d2[u] = j < cnt ? pair_d2<MODE>(p, qp, sh, L, invL) : __int_as_float(0x7fffffff);
      id[u] = __float_as_int(p.w);
    }
  }
}

// Scan one staged source leaf: every (query lane, source point) pair; points at
// or below the lane's running k-th distance are appended to its buffer, and the
// distance list (hence thr) is updated with the oldest kMergeBatch entries once
// a lane has kMergeAt unmerged ones, so that between windows every lane holds
// fewer than kMergeAt (a window adds at most W <= kMergeBatch).  Before a
// compaction every entry is merged: thr is then the k-th smallest distance of
// the whole buffer.  One copy of the candidate code serves every image mode.
template <bool PER, bool LB, int KMAX>
__device__ __forceinline__ void scan_leaf(const float4* __restrict__ sp, int cnt, int G, int sub, int mode,
                                          const float4& qp, const float* sh, float L, float invL,
                                          uint2 (*buf)[32], Cand<KMAX>& C, int k, int lane, bool act,
                                          float lb_d2, int lb_id, Meta* m) {
  constexpr int kCap = L2LWarpSmem<KMAX>::kCap;
  constexpr int W = 8;
  static_assert(kMergeBatch<KMAX> >= W && kMergeAt<KMAX> - 1 <= kMergeBatch<KMAX>,
                "one merge must bring every lane below kMergeAt, a second one to zero");
  for (int j0 = 0; j0 < cnt; j0 += W * G) {
    float d2[W];
    int id[W];
    if (!PER || mode == 0) window_d2<0, W>(sp, j0, cnt, G, sub, qp, sh, L, invL, d2, id);
    else if (mode == 1) window_d2<1, W>(sp, j0, cnt, G, sub, qp, sh, L, invL, d2, id);
    else window_d2<2, W>(sp, j0, cnt, G, sub, qp, sh, L, invL, d2, id);
    float mn = d2[0];
#pragma unroll
    for (int u = 1; u < W; ++u) mn = fminf(mn, d2[u]);
    if (__any_sync(kFull, mn <= C.thr)) {
      // at a window's start C.nb <= kCap - W (the check below compacts
      // otherwise), so the W slots from C.nb on are inside the buffer
#pragma unroll
      for (int u = 0; u < W; ++u) {
        bool keep = d2[u] <= C.thr;
        if (LB) keep = keep && (d2[u] > lb_d2 || (d2[u] == lb_d2 && id[u] > lb_id));
        if (keep) {
          buf[C.nb][lane] = make_uint2(__float_as_uint(d2[u]), (uint32_t)id[u]);
          ++C.nb;
        }
      }
      if (__any_sync(kFull, C.nb - C.nm >= kMergeAt<KMAX> || C.nb > kCap - W)) {
        if (C.nb > kCap) set_error(m, JZT_ERR_INTERNAL, kStageLeaf);  // cannot happen
        merge_distances<KMAX>(buf, C, lane, act);
        if (__any_sync(kFull, C.nb > kCap - W)) {
          if (__any_sync(kFull, C.nb > C.nm)) merge_distances<KMAX>(buf, C, lane, act);
          compact<KMAX>(buf, C, k, lane);
        }
      }
    }
  }
}

// One query leaf: its list's source leaves are staged into shared memory by bulk
// copies, kStages ahead of the computation; the list metadata (source box and
// point range) is read 32 entries at a time, one entry per lane.  Each query
// lane keeps the k smallest distances seen so far in a sorted register list of
// floats, whose last entry is the running k-th distance; every source point at
// or below it is buffered as a (d2, index) pair in the lane's shared-memory
// buffer, and the exact k best (d2, index) keys are selected from that buffer
// once the list is done.  `broken` is set when a bounded wait gave up.
//
// k above 32 runs several passes (LB = true after the first): pass j fills the
// row's columns col0 = 32 j .. col0 + k - 1 (row length k_row) with the k best
// keys strictly above the last key of pass j - 1, read back from the output
// (so exact ties continue in index order).  The interaction lists, built for
// all k_row neighbours, serve every pass.
template <int KMAX, bool PER, bool LB>
__device__ __forceinline__ void l2l_leaf(const L2LArgs& A, int64_t leaf, int64_t nl, L2LWarpSmem<KMAX>& S,
                                         uint32_t& parity, bool& broken, int lane) {
  const float4* __restrict__ pts = A.pts;
  const NodeRec* __restrict__ leaves = A.leaves;
  const uint2* __restrict__ ilo = A.ilo;
  const IEntry* __restrict__ arena = A.arena;
  const float4* __restrict__ qpts = A.qpts;
  const uint2* __restrict__ qrange = A.qrange;
  int32_t* __restrict__ out_idx = A.out_idx;
  float* __restrict__ out_d2 = A.out_d2;
  Meta* m = A.m;
  const int k = A.k, k_row = A.k_row, col0 = A.col0, vec_out = A.vec_out, order = A.order;
  const float L = A.L;
  const float invL = PER ? 1.0f / L : 0.0f;
    const NodeRec me = leaves[leaf];
    // query points of the leaf: the leaf's own points, or (two point sets) its
    // query range; sources are staged from pts by the listed leaves' ranges
    int q = me.count, qfirst = me.first;
    if (qrange) {
      const uint2 qr = qrange[leaf];
      qfirst = (int)qr.x;
      q = (int)qr.y;
    }
    if (q == 0) return;
    int G = 1;
    while (G < 32 && 2 * G * q <= 32) G *= 2;
    const int qi = lane / G, sub = lane & (G - 1);
    const bool act = qi < q;
    const float4 qp = act ? qpts[qfirst + qi] : make_float4(0.f, 0.f, 0.f, 0.f);
    Cand<KMAX> C;
    C.F.init(k, -INFINITY, INFINITY);
    C.nb = C.nm = 0;
    C.thr = act ? INFINITY : -INFINITY;
    C.pushed = 0;
    float lb_d2 = -INFINITY;  // lower bound key (previous pass's last), LB only
    int lb_id = -1;
    if (LB && act) {
      const int64_t row = order == 0 ? (int64_t)__float_as_int(qp.w) : (int64_t)(qfirst + qi);
      lb_d2 = out_d2[row * k_row + col0 - 1];
      lb_id = out_idx[row * k_row + col0 - 1];
    }
    unsigned long long pairs = 0;
    unsigned long long st_examined = 0, st_scanned = 0;
    const uint2 lo = ilo[leaf];
    const uint32_t e_cnt = lo.y & ~kUnsortedBit;
    const bool sorted = (lo.y & kUnsortedBit) == 0;
    const IEntry* list = arena + lo.x;
    bool stop = false;  // sorted list and every later entry beyond all thresholds

    for (uint32_t b0 = 0; b0 < e_cnt && !broken && !stop; b0 += 32) {
      const uint32_t nb = min(32u, e_cnt - b0);
      // metadata of up to 32 entries, one entry per lane, into shared memory:
      // source box (moved to the periodic image chosen for the whole leaf pair),
      // r_low^2, point range and image mode; read back by broadcast loads
      if ((uint32_t)lane < nb) {
        IEntry en = list[b0 + lane];
        if ((uint64_t)(uint32_t)en.src >= (uint64_t)nl) {  // consistency guard
          set_error(m, JZT_ERR_INTERNAL, kStageLeaf);
          en.src = 0;
          en.r2low = INFINITY;
        }
        const NodeRec sr = leaves[en.src];
        float sh[3] = {0.0f, 0.0f, 0.0f};
        const int mode = pair_mode<PER>(me, sr.lo, sr.hi, L, sh);
        float bl[3], bh[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          bl[d] = PER && mode == 1 ? __fadd_rd(sr.lo[d], sh[d]) : sr.lo[d];
          bh[d] = PER && mode == 1 ? __fadd_ru(sr.hi[d], sh[d]) : sr.hi[d];
        }
        S.meta[lane][0] = make_float4(bl[0], bl[1], bl[2], en.r2low);
        S.meta[lane][1] = make_float4(bh[0], bh[1], bh[2], __int_as_float(sr.first));
        S.meta[lane][2] = make_float4(sh[0], sh[1], sh[2], __int_as_float(sr.count | (mode << 8)));
      }
      __syncwarp();
      uint32_t issued = 0, done = 0;
      auto issue = [&](uint32_t e) {
        const float r2 = S.meta[e][0].w;
        if (sorted && !__any_sync(kFull, act && r2 <= C.thr)) {
          stop = true;
          return;
        }
        const int first = __float_as_int(S.meta[e][1].w);
        const int cnt = __float_as_int(S.meta[e][2].w) & 0xff;
        const int st = e % kStages;
        __syncwarp();
        if (lane == 0 && cnt > 0) {  // a source leaf without sources (two point sets) has no copy
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
        const float4 m0 = S.meta[e][0], m1 = S.meta[e][1], m2 = S.meta[e][2];
        const int cnt = __float_as_int(m2.w) & 0xff;
        const int mode = __float_as_int(m2.w) >> 8;
        if (cnt > 0) {
          const bool landed = __all_sync(kFull, mbar_wait(&S.bar[st], (parity >> st) & 1u));
          if (!landed) {
            if (lane == 0) set_error(m, JZT_ERR_TIMEOUT, kStageLeaf);
            broken = true;
            // every copy this warp issued and has not consumed -- the one that
            // timed out included -- must land before the warp leaves
            for (uint32_t r = done; r < issued; ++r) {
              const int s2 = r % kStages;
              if ((__float_as_int(S.meta[r][2].w) & 0xff) > 0) mbar_drain(&S.bar[s2], (parity >> s2) & 1u);
            }
            __syncwarp();
            break;
          }
          parity ^= 1u << st;
          // pad the stage with NaN points (their distances fail every test)
          if (lane >= cnt) S.pts[st][lane] = make_float4(__int_as_float(0x7fffffff), __int_as_float(0x7fffffff),
                                                         __int_as_float(0x7fffffff), __int_as_float(INT_MAX));
        }
        ++done;
        ++st_examined;
        __syncwarp();
        bool skip = !__any_sync(kFull, act && m0.w <= C.thr);
        if (skip && sorted) stop = true;  // r_low only grows along a sorted list
        skip = skip || cnt == 0;          // a leaf without sources is passed over, not a stop
        const float sh[3] = {m2.x, m2.y, m2.z};
        if (!skip) {
          // point-to-box lower bound against this lane's threshold, in the image
          // chosen for the whole leaf pair (all three images when ambiguous)
          const float qq[3] = {qp.x, qp.y, qp.z};
          const float bl[3] = {m0.x, m0.y, m0.z}, bh[3] = {m1.x, m1.y, m1.z};
          float pb = 0.0f;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float g = PER && mode == 2
                                ? gap_rd_per(qq[d], qq[d], bl[d], bh[d], L)
                                : fmaxf(0.0f, fmaxf(__fsub_rd(bl[d], qq[d]), __fsub_rd(qq[d], bh[d])));
            pb = __fmaf_rd(g, g, pb);
          }
          skip = !__any_sync(kFull, act && pb * kLowSlack <= C.thr);
        }
        if (!skip) {
          pairs += (unsigned long long)q * (unsigned long long)cnt;
          ++st_scanned;
          scan_leaf<PER, LB, KMAX>(S.pts[st], cnt, G, sub, mode, qp, sh, L, invL, S.buf, C, k, lane, act,
                                   lb_d2, lb_id, m);
        }
        __syncwarp();
        if (!stop && issued < nb) issue(issued);
      }
    }
    // final k-th distance (fewer than kMergeAt entries are unmerged here), drop the
    // entries beyond it, exact (d2, index) selection
    merge_distances<KMAX>(S.buf, C, lane, act);
    compact<KMAX>(S.buf, C, k, lane);
    // after the compaction a lane's buffer holds at most KMAX entries, the k best
    // of the lane's sources among them; one descending sorting network puts them,
    // smallest last, in the last slots (pads of kKeyInf in front)
    unsigned long long v[KMAX];
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
      const uint2 e = S.buf[i][lane];
      v[i] = i < C.nb ? (((unsigned long long)e.x << 32) | (e.y + 1u)) : kKeyInf;
    }
    sort_desc<KMAX>(v);
    if (G == 1) {  // one lane per query: the row is written straight from the network's registers
      if (act && !broken) {
        const int64_t row = order == 0 ? (int64_t)__float_as_int(qp.w) : (int64_t)(qfirst + qi);
        int32_t* oi = out_idx + row * k_row + col0;
        float* od = out_d2 + row * k_row + col0;
        if (vec_out && k == KMAX) {  // whole rows as 16-byte stores; j-th best in v[KMAX - 1 - j]
#pragma unroll
          for (int e = 0; e < KMAX; e += 4) {
            const unsigned long long a0 = v[KMAX - 1 - e], a1 = v[KMAX - 2 - e], a2 = v[KMAX - 3 - e],
                                     a3 = v[KMAX - 4 - e];
            reinterpret_cast<int4*>(oi)[e / 4] =
                make_int4((int32_t)(uint32_t)(a0 & 0xffffffffull) - 1, (int32_t)(uint32_t)(a1 & 0xffffffffull) - 1,
                          (int32_t)(uint32_t)(a2 & 0xffffffffull) - 1, (int32_t)(uint32_t)(a3 & 0xffffffffull) - 1);
            reinterpret_cast<float4*>(od)[e / 4] =
                make_float4(__uint_as_float((uint32_t)(a0 >> 32)), __uint_as_float((uint32_t)(a1 >> 32)),
                            __uint_as_float((uint32_t)(a2 >> 32)), __uint_as_float((uint32_t)(a3 >> 32)));
          }
        } else {
#pragma unroll
          for (int e = 0; e < KMAX; ++e) {
            if (e >= KMAX - k) {
              oi[KMAX - 1 - e] = (int32_t)(uint32_t)(v[e] & 0xffffffffull) - 1;
              od[KMAX - 1 - e] = __uint_as_float((uint32_t)(v[e] >> 32));
            }
          }
        }
      }
    } else {
      // G lanes per query: each sub-lane's list (ascending, kKeyInf pads last) is
      // merged with its partners' (butterfly), keeping the KMAX smallest keys
      RegTopK<unsigned long long, KMAX> T;
#pragma unroll
      for (int e = 0; e < KMAX; ++e) T.t[e] = v[KMAX - 1 - e];
      for (int st = 1; st < G; st <<= 1) {
        unsigned long long pb[KMAX];
#pragma unroll
        for (int e = 0; e < KMAX; ++e) pb[e] = __shfl_xor_sync(kFull, T.t[e], st);
        T.template merge<KMAX>(pb);
      }
      if (act && sub == 0 && !broken) {
        const int64_t row = order == 0 ? (int64_t)__float_as_int(qp.w) : (int64_t)(qfirst + qi);
        int32_t* oi = out_idx + row * k_row + col0;
        float* od = out_d2 + row * k_row + col0;
#pragma unroll
        for (int e = 0; e < KMAX; ++e) {
          if (e < k) {
            oi[e] = (int32_t)(uint32_t)(T.t[e] & 0xffffffffull) - 1;
            od[e] = __uint_as_float((uint32_t)(T.t[e] >> 32));
          }
        }
      }
    }
    if (lane == 0 && pairs) {
      atomicAdd(&m->knn_pairs, pairs);
      atomicAdd(&m->knn_stats[0], st_examined);
      atomicAdd(&m->knn_stats[1], st_scanned);
    }
    {
      unsigned long long a = C.pushed;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
      if (lane == 0) atomicAdd(&m->knn_stats[2], a);
    }
    __syncwarp();
}

// One warp per query leaf, leaves taken in order from the tree's counter `ctr`.
template <int KMAX, bool PER, bool LB>
__global__ void __launch_bounds__(32 * kL2LWarps, JZT_L2L_MINBLOCKS(KMAX)) k_l2l_knn(L2LArgs A, int ctr) {
  extern __shared__ __align__(16) unsigned char l2l_smem[];
  Meta* m = A.m;
  if (warp_failed(m)) return;
  const int w = warp_id(), lane = lane_id();
  L2LWarpSmem<KMAX>& S = reinterpret_cast<L2LWarpSmem<KMAX>*>(l2l_smem)[w];
  if (lane == 0) {
    for (int t = 0; t < kStages; ++t) mbar_init(&S.bar[t], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  uint32_t parity = 0;  // bit t: parity of the next completion of stage t
  const int64_t nl = m->n_nodes[0];
  bool broken = false;
  while (!broken) {
    int64_t leaf = 0;
    if (lane == 0) leaf = atomicAdd(&m->tile_ctr[ctr], 1u);
    leaf = __shfl_sync(kFull, leaf, 0);
    if (leaf >= nl) break;
    l2l_leaf<KMAX, PER, LB>(A, leaf, nl, S, parity, broken, lane);
  }
}

// Batches: the LeafToLeaf work of many trees (jobs of one k class and one kind
// of boundary) as one persistent launch over a device work queue.  Item i of
// the queue is leaf i - prefix[j] of job j, prefix[j] <= i < prefix[j + 1] (the
// jobs' leaf counts, summed on the device once their trees exist); every warp
// pops the next item from the shared counter until the queue is empty.  Jobs
// whose status is already an error are passed over.
template <int KMAX, bool PER>
__global__ void __launch_bounds__(32 * kL2LWarps, JZT_L2L_MINBLOCKS(KMAX))
    k_l2l_knn_queue(const L2LArgs* __restrict__ jobs, const int64_t* __restrict__ prefix, int n_jobs,
                    unsigned long long* next) {
  extern __shared__ __align__(16) unsigned char l2l_smem[];
  const int w = warp_id(), lane = lane_id();
  L2LWarpSmem<KMAX>& S = reinterpret_cast<L2LWarpSmem<KMAX>*>(l2l_smem)[w];
  if (lane == 0) {
    for (int t = 0; t < kStages; ++t) mbar_init(&S.bar[t], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  uint32_t parity = 0;
  const int64_t total = prefix[n_jobs];
  bool broken = false;
  while (!broken) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(next, 1ull);
    item = __shfl_sync(kFull, item, 0);
    if ((int64_t)item >= total) break;
    int lo = 0, hi = n_jobs - 1;  // the job: largest j with prefix[j] <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= (int64_t)item) lo = mid;
      else hi = mid - 1;
    }
    const L2LArgs A = jobs[lo];
    if (warp_failed(A.m)) continue;
    l2l_leaf<KMAX, PER, false>(A, (int64_t)item - prefix[lo], prefix[lo + 1] - prefix[lo], S, parity, broken, lane);
  }
}

// Interaction-list entries written by one plane's NodeToNode (arena growth).
__global__ void k_plane_mark(Meta* m, int plane, int end) {
  if (threadIdx.x != 0) return;
  if (!end) m->tile_ctr[kCtrN2N] = 0;  // the plane's NodeToNode takes its parents from here
  else m->tile_ctr[kCtrLists] = 0;    // the list sort that follows takes its lists from here
  if (!end) m->knn_plane_entries[plane] = m->arena_used;
  else m->knn_plane_entries[plane] = m->arena_used - m->knn_plane_entries[plane];
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
  const NodeRec* par_nodes = (p + 1 < L.n_planes) ? at<NodeRec>(ws, L.nodes[p + 1]) : nullptr;
  const float* rint = p >= 1 ? at<float>(ws, L.rint[p]) : nullptr;
  k_n2n_knn<NR, PER><<<grid_for(L.cap_nodes[p + 1] * 32, 32 * kN2NWarps, sms * 16), 32 * kN2NWarps, 0, s>>>(
      at<int32_t>(ws, L.spl[p + 1]), at<uint2>(ws, L.ilo[p + 1]), par_nodes, at<NodeRec>(ws, L.nodes[p]), rint,
      at<uint2>(ws, L.ilo[p]), at<IEntry>(ws, L.arena), p + 1, k, pl, L.cap_ilist,
      (int64_t)L.total, m); note_launch();
}

template <int KMAX, bool PER, bool LB>
void l2l_knn(const Layout& L, char* ws, int k, int k_row, int col0, int pass, float pl, int order,
             int32_t* idx, float* d2, cudaStream_t s) {
  Meta* m = at<Meta>(ws, L.meta);
  const int sms = 152;
  const size_t smem = sizeof(L2LWarpSmem<KMAX>) * kL2LWarps;
  cudaFuncSetAttribute(k_l2l_knn<KMAX, PER, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // two point sets: sources pts2[0, n_src), queries pts2[n_src, n) with per-leaf ranges
  const bool sets = L.n_src < L.n;
  const float4* src = sets ? at<float4>(ws, L.pts2) : at<float4>(ws, L.pts);
  const float4* qry = sets ? src + L.n_src : src;
  const uint2* qrange = sets ? at<uint2>(ws, L.qrange) : nullptr;
  // 16-byte row stores need 16-byte aligned outputs and rows of a multiple of 4 entries
  // (col0 is a multiple of 32)
  const int vec_out = ((reinterpret_cast<uintptr_t>(idx) | reinterpret_cast<uintptr_t>(d2)) & 15u) == 0 &&
                      (k_row % 4) == 0;
  L2LArgs A;
  A.pts = src;
  A.leaves = at<NodeRec>(ws, L.nodes[0]);
  A.ilo = at<uint2>(ws, L.ilo[0]);
  A.arena = at<IEntry>(ws, L.arena);
  A.qpts = qry;
  A.qrange = qrange;
  A.out_idx = idx;
  A.out_d2 = d2;
  A.m = m;
  A.k = k;
  A.k_row = k_row;
  A.col0 = col0;
  A.vec_out = vec_out;
  A.order = order;
  A.L = pl;
  k_l2l_knn<KMAX, PER, LB><<<sms * 8, 32 * kL2LWarps, smem, s>>>(A, kCtrWalk + pass); note_launch();
}

// Everything of the kNN walk before the LeafToLeaf: the top level, the internal
// radius bounds and NodeToNode + list sort per plane.
template <bool PER>
void knn_prepare(const Layout& L, char* ws, float pl, int k, cudaStream_t s) {
  Meta* m = at<Meta>(ws, L.meta);
  const int sms = 152;
  const int P = L.n_planes;
  prof_begin(kPhKnnTop, s);
  k_walk_reset<<<1, 32, 0, s>>>(m); note_launch();
  launch_super_level(L, ws, s);
  k_dense_ilist<<<grid_for(L.cap_nodes[P], 128, sms * 4), 128, 0, s>>>(
      m, at<uint2>(ws, L.ilo[P]), at<IEntry>(ws, L.arena), P, 0, L.cap_ilist, m); note_launch();
  for (int p = 1; p < P; ++p) {
    const float* rc = p >= 2 ? at<float>(ws, L.rint[p - 1]) : nullptr;
    k_internal_bounds<8, PER><<<grid_for(L.cap_nodes[p] * 32, 128, sms * 16), 128, 0, s>>>(
        at<int32_t>(ws, L.spl[p]), at<NodeRec>(ws, L.nodes[p - 1]), rc, at<float>(ws, L.rint[p]), p, k, pl,
        m); note_launch();
  }
  prof_end(kPhKnnTop, s);
  for (int p = P - 1; p >= 0; --p) {
    prof_begin(kPhKnnN2N, s);
    k_plane_mark<<<1, 32, 0, s>>>(m, p, 0); note_launch();
    if (L.heap <= 4) n2n_knn_plane<4, PER>(L, ws, p, k, pl, s);
    else if (L.heap <= 8) n2n_knn_plane<8, PER>(L, ws, p, k, pl, s);
    else n2n_knn_plane<16, PER>(L, ws, p, k, pl, s);
    k_plane_mark<<<1, 32, 0, s>>>(m, p, 1); note_launch();
    prof_end(kPhKnnN2N, s);
    prof_begin(kPhKnnSort, s);
    k_sort_lists<<<grid_for(L.cap_nodes[p] * 32, 128, sms * 16), 128, 0, s>>>(
        at<uint2>(ws, L.ilo[p]), at<IEntry>(ws, L.arena), p, m); note_launch();
    prof_end(kPhKnnSort, s);
  }
  k_walk_peak<<<1, 32, 0, s>>>(m); note_launch();
}

template <bool PER>
void knn_all(const Layout& L, char* ws, float pl, int k, int order, int32_t* idx, float* d2,
             cudaStream_t s) {
  knn_prepare<PER>(L, ws, pl, k, s);
  prof_begin(kPhKnnL2L, s);
  if (k <= 4) l2l_knn<4, PER, false>(L, ws, k, k, 0, 0, pl, order, idx, d2, s);
  else if (k <= 8) l2l_knn<8, PER, false>(L, ws, k, k, 0, 0, pl, order, idx, d2, s);
  else if (k <= 16) l2l_knn<16, PER, false>(L, ws, k, k, 0, 0, pl, order, idx, d2, s);
  else if (k <= kMaxK) l2l_knn<32, PER, false>(L, ws, k, k, 0, 0, pl, order, idx, d2, s);
  else
    for (int c0 = 0, pass = 0; c0 < k; c0 += kMaxK, ++pass) {  // k / 32 passes (at most 8 counters)
      const int kp = k - c0 < kMaxK ? k - c0 : kMaxK;
      if (c0 == 0) l2l_knn<32, PER, false>(L, ws, kp, k, c0, pass, pl, order, idx, d2, s);
      else l2l_knn<32, PER, true>(L, ws, kp, k, c0, pass, pl, order, idx, d2, s);
    }
  prof_end(kPhKnnL2L, s);
}

// Leaf counts of the queued jobs (0 for a job whose status is an error) summed
// into prefix[0..n]; the queue counter starts at 0.  One block.
__global__ void __launch_bounds__(1024) k_queue_prefix(const L2LArgs* __restrict__ jobs, int n, int64_t* prefix,
                                                       unsigned long long* next) {
  __shared__ int64_t s_w[32];
  __shared__ int64_t s_carry;
  if (threadIdx.x == 0) {
    s_carry = 0;
    *next = 0ull;
    prefix[0] = 0;
  }
  __syncthreads();
  for (int b = 0; b < n; b += 1024) {
    const int j = b + threadIdx.x;
    int64_t v = 0;
    if (j < n) {
      const Meta* m = jobs[j].m;
      v = failed(m) ? 0 : (int64_t)m->n_nodes[0];
    }
    int64_t inc = v;  // inclusive scan: warps, then warp totals
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(kFull, inc, o);
      if (lane_id() >= o) inc += t;
    }
    if (lane_id() == 31) s_w[warp_id()] = inc;
    __syncthreads();
    if (warp_id() == 0) {
      int64_t wv = s_w[lane_id()];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, wv, o);
        if (lane_id() >= o) wv += t;
      }
      s_w[lane_id()] = wv;
    }
    __syncthreads();
    const int64_t before = s_carry + (warp_id() > 0 ? s_w[warp_id() - 1] : 0);
    if (j < n) prefix[j + 1] = before + inc;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += s_w[31];
    __syncthreads();
  }
}

// Status word of every queued job into the caller's job-status array.
__global__ void k_queue_statuses(const L2LArgs* __restrict__ jobs, int n, int32_t* status) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    status[jobs[j].job] = *reinterpret_cast<const volatile int32_t*>(&jobs[j].m->status);
}

// Copies up to kArgsPerLaunch job descriptors, passed by value, to the device.
constexpr int kArgsPerLaunch = 16;
struct ArgsChunk {
  L2LArgs a[kArgsPerLaunch];
};
__global__ void k_put_args(ArgsChunk c, int count, L2LArgs* dst) {
  if ((int)threadIdx.x < count) dst[threadIdx.x] = c.a[threadIdx.x];
}

template <int KMAX, bool PER>
void queue_launch(const L2LArgs* d_jobs, const int64_t* d_prefix, int n_jobs, unsigned long long* d_next,
                  cudaStream_t s) {
  const size_t smem = sizeof(L2LWarpSmem<KMAX>) * kL2LWarps;
  cudaFuncSetAttribute(k_l2l_knn_queue<KMAX, PER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_l2l_knn_queue<KMAX, PER><<<152 * JZT_L2L_MINBLOCKS(KMAX), 32 * kL2LWarps, smem, s>>>(d_jobs, d_prefix, n_jobs,
                                                                                        d_next);
  note_launch();
}

}  // namespace

namespace {

__global__ void k_selftest_reset(Meta* m, uint32_t* flag) {
  if (threadIdx.x == 0) {
    m->status = 0;
    m->detail = 0;
    *flag = 0;
  }
}

// Failure-path self-test: the bounded waits of the walk and the sort, made to
// run out -- an mbarrier phase that never completes (nobody arrives) and a
// published-word flag that nobody sets.  Both must end with JZT_ERR_TIMEOUT in
// the status word and leave the context usable.
__global__ void k_selftest_wait(int which, long long limit, const uint32_t* flag, Meta* m) {
  __shared__ uint64_t bar;
  const int lane = lane_id();
  if (lane == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (which == 0) {
    const bool ok = __all_sync(kFull, mbar_wait_n(&bar, 0u, limit));
    if (!ok && lane == 0) set_error(m, JZT_ERR_TIMEOUT, kStageLeaf);
  } else if (lane == 0) {
    long long it = 0;
    while (ld_relaxed_u32(flag) == 0u && ++it < limit) {
    }
    if (it >= limit) set_error(m, JZT_ERR_TIMEOUT, kStageSort);
  }
}

}  // namespace

void launch_selftest_wait(const Layout& L, char* ws, int which, long long limit, cudaStream_t s) {
  Meta* m = at<Meta>(ws, L.meta);
  uint32_t* flag = at<uint32_t>(ws, L.arena);
  k_selftest_reset<<<1, 32, 0, s>>>(m, flag); note_launch();
  k_selftest_wait<<<1, 32, 0, s>>>(which, limit, flag, m); note_launch();
}

void launch_knn_prepare(const Layout& L, char* ws, float periodic_L, int k, cudaStream_t s) {
  if (periodic_L > 0.0f) knn_prepare<true>(L, ws, periodic_L, k, s);
  else knn_prepare<false>(L, ws, 0.0f, k, s);
}

void make_l2l_args(const Layout& L, char* ws, float periodic_L, int k, int32_t* d_idx, float* d_d2, int job,
                   L2LArgs* out) {
  L2LArgs A;
  std::memset(&A, 0, sizeof(A));
  A.pts = at<float4>(ws, L.pts);
  A.leaves = at<NodeRec>(ws, L.nodes[0]);
  A.ilo = at<uint2>(ws, L.ilo[0]);
  A.arena = at<IEntry>(ws, L.arena);
  A.qpts = A.pts;
  A.qrange = nullptr;
  A.out_idx = d_idx;
  A.out_d2 = d_d2;
  A.m = at<Meta>(ws, L.meta);
  A.k = k;
  A.k_row = k;
  A.col0 = 0;
  A.vec_out = ((reinterpret_cast<uintptr_t>(d_idx) | reinterpret_cast<uintptr_t>(d_d2)) & 15u) == 0 && (k % 4) == 0;
  A.order = 0;
  A.L = periodic_L > 0.0f ? periodic_L : 0.0f;
  A.job = job;
  *out = A;
}

int queue_kmax(int k) { return k <= 4 ? 4 : (k <= 8 ? 8 : (k <= 16 ? 16 : 32)); }

void launch_put_args(const L2LArgs* h_args, int n, L2LArgs* d_args, cudaStream_t s) {
  for (int b = 0; b < n; b += kArgsPerLaunch) {
    ArgsChunk c;
    const int cnt = n - b < kArgsPerLaunch ? n - b : kArgsPerLaunch;
    for (int i = 0; i < cnt; ++i) c.a[i] = h_args[b + i];
    k_put_args<<<1, 32, 0, s>>>(c, cnt, d_args + b);
    note_launch();
  }
}

void launch_knn_queue(int kmax, bool periodic, const L2LArgs* d_jobs, int n_jobs, int64_t* d_prefix,
                      unsigned long long* d_next, int32_t* d_job_status, cudaStream_t s) {
  if (n_jobs <= 0) return;
  k_queue_prefix<<<1, 1024, 0, s>>>(d_jobs, n_jobs, d_prefix, d_next); note_launch();
  prof_begin(kPhKnnL2L, s);
  if (periodic) {
    if (kmax == 4) queue_launch<4, true>(d_jobs, d_prefix, n_jobs, d_next, s);
    else if (kmax == 8) queue_launch<8, true>(d_jobs, d_prefix, n_jobs, d_next, s);
    else if (kmax == 16) queue_launch<16, true>(d_jobs, d_prefix, n_jobs, d_next, s);
    else queue_launch<32, true>(d_jobs, d_prefix, n_jobs, d_next, s);
  } else {
    if (kmax == 4) queue_launch<4, false>(d_jobs, d_prefix, n_jobs, d_next, s);
    else if (kmax == 8) queue_launch<8, false>(d_jobs, d_prefix, n_jobs, d_next, s);
    else if (kmax == 16) queue_launch<16, false>(d_jobs, d_prefix, n_jobs, d_next, s);
    else queue_launch<32, false>(d_jobs, d_prefix, n_jobs, d_next, s);
  }
  prof_end(kPhKnnL2L, s);
  k_queue_statuses<<<(n_jobs + 255) / 256, 256, 0, s>>>(d_jobs, n_jobs, d_job_status); note_launch();
}

void launch_knn(const Layout& L, char* ws, float periodic_L, int k, int order, int32_t* d_idx,
                float* d_d2, cudaStream_t s) {
  if (periodic_L > 0.0f) knn_all<true>(L, ws, periodic_L, k, order, d_idx, d_d2, s);
  else knn_all<false>(L, ws, 0.0f, k, order, d_idx, d_d2, s);
}

}  // namespace jzt
