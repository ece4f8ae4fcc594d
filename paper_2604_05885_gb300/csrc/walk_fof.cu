// Friends-of-friends on the plane hierarchy (Sec. IV-A).
//
// Group pointers igroup (a root points to itself, any other entry to a smaller
// index of its group) live on every plane and on the points.  Per plane, from
// the top down:
//   NodeToNode -- every interacting child pair (i, j): discard if already in one
//                 group or d_low > b; link the two nodes whole if d_up <= b (every
//                 cross pair is within b); otherwise keep the pair for the next
//                 plane.  Links are lock-free CAS unions (higher root -> lower).
//   Contract   -- every pointer to its root.
//   ParentToNode -- children of a linked parent point to the first child of the
//                 parent's root; others start as their own roots, self-linked
//                 when their diagonal is <= b.
// LeafToLeaf links point pairs with d2 <= b^2; a final contraction gives the
// roots; each group is labelled with its smallest original index.
//
// Interactions are kept as pair lists (i <= j, each unordered pair once) in the
// arena; a warp stages the pairs it keeps in shared memory and reserves their
// range with one atomic.
#include <cuda_runtime.h>


#include "common.cuh"

namespace jzt {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFofWarps = 4;
constexpr int kPairBuf = 256;  // staged pairs per warp

__global__ void k_fof_reset(Meta* m) {
  if (threadIdx.x == 0) {
    m->arena_used = 0;
    m->arena_peak = 0;
    m->fof_pairs = 0;
  }
  if (threadIdx.x < kMaxPlanes + 1) {
    m->pair_off[threadIdx.x] = 0;
    m->pair_cnt[threadIdx.x] = 0;
  }
  if (threadIdx.x >= kCtrWalk && threadIdx.x < 32) m->tile_ctr[threadIdx.x] = 0;
}

// Super-node pairs (S, T), T >= S (Alg. 1's dense list, each unordered pair once).
__global__ void k_fof_super_pairs(int2* pairs, int sup_plane, int64_t cap, int64_t ws_total,
                                  Meta* m) {
  if (failed(m)) return;
  const int64_t ns = m->n_nodes[sup_plane];
  const int64_t total = ns * (ns + 1) / 2;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    m->pair_off[sup_plane] = 0;
    m->pair_cnt[sup_plane] = (unsigned long long)total;
    m->arena_used = (unsigned long long)total;
    if (total > cap) {
      set_error(m, JZT_ERR_CAPACITY, kStageTop);
      atomicMax(reinterpret_cast<unsigned long long*>(&m->required_bytes),
                (unsigned long long)(ws_total + (total - cap) * 8));
    }
  }
  if (total > cap) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t off = i * ns - i * (i - 1) / 2;
    for (int64_t j = i; j < ns; ++j) pairs[off + (j - i)] = make_int2((int)i, (int)j);
  }
}

// Top plane: every node its own root; self-linked when its diagonal is <= b.
__global__ void k_fof_init_top(const NodeRec* __restrict__ nodes, int32_t* ig, uint8_t* lk,
                               int plane, float L, float b2, const Meta* m) {
  if (failed(m)) return;
  const int64_t nn = m->n_nodes[plane];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    const NodeRec r = nodes[i];
    const float d2 = L > 0.0f ? box_dup2<true>(r.lo, r.hi, r.lo, r.hi, L)
                              : box_dup2<false>(r.lo, r.hi, r.lo, r.hi, L);
    ig[i] = (int32_t)i;
    lk[i] = d2 <= b2 ? 1 : 0;
  }
}

__global__ void k_mark_plane_start(Meta* m, int plane) {
  if (threadIdx.x == 0) m->pair_off[plane] = m->arena_used;
}
__global__ void k_mark_plane_end(Meta* m, int plane) {
  if (threadIdx.x == 0) {
    unsigned long long used = m->arena_used;
    m->pair_cnt[plane] = used - m->pair_off[plane];
    if (used > m->arena_peak) m->arena_peak = used;
  }
}

// Flush a warp's staged pairs to the arena (one atomic per flush).
__device__ __forceinline__ void flush_pairs(int2* s_buf, int& nbuf, int2* arena, int64_t cap,
                                            int64_t ws_total, Meta* m) {
  const int lane = lane_id();
  if (nbuf == 0) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&m->arena_used, (unsigned long long)nbuf);
  base = __shfl_sync(kFull, base, 0);
  if (base + nbuf > (unsigned long long)cap) {
    if (lane == 0) {
      set_error(m, JZT_ERR_CAPACITY, kStageFof);
      atomicMax(reinterpret_cast<unsigned long long*>(&m->required_bytes),
                (unsigned long long)(ws_total + (int64_t)(base + nbuf - cap) * 8));
    }
  } else {
    for (int t = lane; t < nbuf; t += 32) arena[base + t] = s_buf[t];
  }
  __syncwarp();
  nbuf = 0;
}

template <bool PER>
__global__ void __launch_bounds__(32 * kFofWarps) k_n2n_fof(
    const int32_t* __restrict__ spl_par, const NodeRec* __restrict__ nodes, int32_t* ig, uint8_t* lk,
    int2* arena, int par_plane, float L, float b2, int64_t cap, int64_t ws_total, Meta* m) {
  __shared__ int2 s_buf[kFofWarps][kPairBuf];
  if (warp_failed(m)) return;
  const int w = warp_id(), lane = lane_id();
  const unsigned long long in_off = m->pair_off[par_plane];
  const int64_t n_in = (int64_t)m->pair_cnt[par_plane];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int nbuf = 0;
  bool union_fail = false;
  const int64_t npar = m->n_nodes[par_plane];
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < n_in; t += nw) {
    const int2 pr = arena[in_off + t];
    if ((uint64_t)(uint32_t)pr.x >= (uint64_t)npar || (uint64_t)(uint32_t)pr.y >= (uint64_t)npar) {
      if (lane == 0) set_error(m, JZT_ERR_INTERNAL, kStageFof);  // consistency guard
      continue;
    }
    const int a0 = spl_par[pr.x], a1 = spl_par[pr.x + 1];
    const int b0 = spl_par[pr.y], b1 = spl_par[pr.y + 1];
    const int Ca = a1 - a0, Cb = b1 - b0;
    const bool self = pr.x == pr.y;
    const int total = Ca * Cb;
    for (int u0 = 0; u0 < total; u0 += 32) {
      const int u = u0 + lane;
      bool keep = false;
      int i = 0, j = 0;
      if (u < total) {
        i = a0 + u / Cb;
        j = b0 + u % Cb;
        if (!(self && j < i)) {
          if (i == j) {
            keep = lk[i] == 0;
          } else {
            const NodeRec ri = nodes[i], rj = nodes[j];
            const float dl = box_dlow2<PER>(ri.lo, ri.hi, rj.lo, rj.hi, L);
            if (dl <= b2) {
              const float du = box_dup2<PER>(ri.lo, ri.hi, rj.lo, rj.hi, L);
              if (du <= b2) {
                if (!uf_union(ig, i, j)) union_fail = true;
                lk[i] = 1;
                lk[j] = 1;
              } else {
                keep = uf_find(ig, i) != uf_find(ig, j);
              }
            }
          }
        }
      }
      const unsigned bal = __ballot_sync(kFull, keep);
      const int nk = __popc(bal);
      if (nbuf + nk > kPairBuf) flush_pairs(s_buf[w], nbuf, arena, cap, ws_total, m);
      if (keep) s_buf[w][nbuf + __popc(bal & ((1u << lane) - 1u))] = make_int2(i, j);
      nbuf += nk;
      __syncwarp();
    }
  }
  flush_pairs(s_buf[w], nbuf, arena, cap, ws_total, m);
  if (__any_sync(kFull, union_fail) && lane == 0) set_error(m, JZT_ERR_TIMEOUT, kStageFof);
}

__global__ void k_contract(int32_t* ig, int plane, int64_t n_fixed, const Meta* m) {
  if (failed(m)) return;
  const int64_t nn = plane >= 0 ? (int64_t)m->n_nodes[plane] : n_fixed;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x)
    ig[i] = uf_root_ro(ig, (int)i);
}

// Plane p -> p-1 (Eq. igroup): one warp per parent.
template <bool PER>
__global__ void k_parent_to_node(const int32_t* __restrict__ spl, const int32_t* __restrict__ ig_par,
                                 const uint8_t* __restrict__ lk_par,
                                 const NodeRec* __restrict__ child, int32_t* ig, uint8_t* lk,
                                 int par_plane, float L, float b2, const Meta* m) {
  if (warp_failed(m)) return;
  const int64_t np = m->n_nodes[par_plane];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t P = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; P < np; P += nw) {
    const int R = ig_par[P];
    const bool linked = lk_par[P] != 0;
    const int first = spl[R];
    const int c0 = spl[P], c1 = spl[P + 1];
    for (int c = c0 + lane_id(); c < c1; c += 32) {
      if (linked) {
        ig[c] = first;
        lk[c] = 1;
      } else {
        const NodeRec r = child[c];
        ig[c] = c;
        lk[c] = box_dup2<PER>(r.lo, r.hi, r.lo, r.hi, L) <= b2 ? 1 : 0;
      }
    }
  }
}

// Leaves -> points.
__global__ void k_leaf_to_points(const int32_t* __restrict__ spl0, const int32_t* __restrict__ ig0,
                                 const uint8_t* __restrict__ lk0, int32_t* ig_pt, const Meta* m) {
  if (warp_failed(m)) return;
  const int64_t nl = m->n_nodes[0];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t Lf = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; Lf < nl; Lf += nw) {
    const int R = ig0[Lf];
    const bool linked = lk0[Lf] != 0;
    const int first = spl0[R];
    const int s0 = spl0[Lf], s1 = spl0[Lf + 1];
    for (int a = s0 + lane_id(); a < s1; a += 32) ig_pt[a] = linked ? first : a;
  }
}

__device__ __forceinline__ float wrap1(float d, float L, float invL) {
  return d - L * rintf(d * invL);
}

// Leaf pairs: link every point pair with float32 d2 <= b^2.
template <bool PER>
__global__ void __launch_bounds__(128) k_l2l_fof(const float4* __restrict__ pts,
                                                 const NodeRec* __restrict__ leaves,
                                                 const int2* __restrict__ arena, int32_t* ig_pt,
                                                 float L, float b2, Meta* m) {
  __shared__ float4 s_b[128 / 32][32];  // per warp: the source leaf's points (leaves hold <= 32)
  if (failed(m)) return;
  const unsigned long long off = m->pair_off[0];
  const int64_t np = (int64_t)m->pair_cnt[0];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = lane_id();
  float4* sb = s_b[warp_id()];
  const float invL = PER ? 1.0f / L : 0.0f;
  const float halfL = 0.5f * L;
  bool union_fail = false;
  unsigned long long pairs = 0;
  const int64_t nl = m->n_nodes[0];
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < np; t += nw) {
    const int2 pr = arena[off + t];
    if ((uint64_t)(uint32_t)pr.x >= (uint64_t)nl || (uint64_t)(uint32_t)pr.y >= (uint64_t)nl) {
      if (lane == 0) set_error(m, JZT_ERR_INTERNAL, kStageFof);  // consistency guard
      continue;
    }
    const NodeRec A = leaves[pr.x], B = leaves[pr.y];
    const bool self = pr.x == pr.y;
    pairs += self ? (unsigned long long)A.count * (A.count - 1) / 2
                  : (unsigned long long)A.count * B.count;
    float sh[3] = {0.f, 0.f, 0.f};
    bool ambiguous = false;
    if (PER) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float dlo = __fsub_rd(B.lo[d], A.hi[d]);
        const float dhi = __fsub_ru(B.hi[d], A.lo[d]);
        if (dlo >= -halfL && dhi <= halfL) sh[d] = 0.0f;
        else if (dlo >= halfL) sh[d] = -L;
        else if (dhi <= -halfL) sh[d] = L;
        else ambiguous = true;
      }
    }
    // the source points in shared memory (one coalesced load; leaves hold at most
    // 32 points -- larger ranges are read from global memory)
    const bool staged = B.count <= 32;
    __syncwarp();
    if (staged && lane < B.count) sb[lane] = pts[B.first + lane];
    __syncwarp();
    constexpr int U = 4;  // source points per step, the union only on a hit
    if (self && staged) {
      // a leaf with itself: lane a takes the partners (a + d) mod c, d = 1 .. c/2
      // (d = c/2 of an even c from the lower half only), so every unordered pair
      // is tested exactly once and the lanes share the triangle evenly.  d^2
      // does not depend on the pair's orientation: the differences only change
      // sign (the image shift of a leaf with itself is zero or the minimum image).
      const int c = A.count, half = c / 2;
      const bool act = lane < c;
      const float4 pa = act ? sb[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int d0 = 1; d0 <= half; d0 += U) {
        float d2[U];
        int pb_i[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int d = d0 + u;
          int bi = lane + d;
          if (bi >= c) bi -= c;
          const bool ok = act && d <= half && !(2 * d == c && lane >= half);
          pb_i[u] = ok ? bi : 0;
          const float4 pb = sb[pb_i[u]];
          float dx = pb.x - pa.x, dy = pb.y - pa.y, dz = pb.z - pa.z;
          if (PER && ambiguous) {
            dx = wrap1(dx, L, invL);
            dy = wrap1(dy, L, invL);
            dz = wrap1(dz, L, invL);
          }
          d2[u] = ok ? __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) : INFINITY;
        }
        const bool any = d2[0] <= b2 || d2[1] <= b2 || d2[2] <= b2 || d2[3] <= b2;
        if (any) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (d2[u] <= b2 && !uf_union(ig_pt, A.first + lane, A.first + pb_i[u])) union_fail = true;
        }
      }
      continue;
    }
    for (int a0 = 0; a0 < A.count; a0 += 32) {
      const int ia = a0 + lane;
      const bool act = ia < A.count;
      const int a = A.first + ia;
      const float4 pa = act ? pts[a] : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int jb0 = self ? a0 : 0; jb0 < B.count; jb0 += U) {
        float d2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int jb = jb0 + u;
          const int jc = jb < B.count ? jb : B.count - 1;
          const float4 pb = staged ? sb[jc] : __ldg(pts + B.first + jc);
          float dx = pb.x - pa.x, dy = pb.y - pa.y, dz = pb.z - pa.z;
          if (PER) {
            if (ambiguous) {
              dx = wrap1(dx, L, invL);
              dy = wrap1(dy, L, invL);
              dz = wrap1(dz, L, invL);
            } else {
              dx = __fadd_rn(dx, sh[0]);
              dy = __fadd_rn(dy, sh[1]);
              dz = __fadd_rn(dz, sh[2]);
            }
          }
          d2[u] = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
          const int bb = B.first + jb;
          if (!act || jb >= B.count || (self && bb <= a)) d2[u] = INFINITY;
        }
        const bool any = d2[0] <= b2 || d2[1] <= b2 || d2[2] <= b2 || d2[3] <= b2;
        if (any) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (d2[u] <= b2 && !uf_union(ig_pt, a, B.first + jb0 + u)) union_fail = true;
        }
      }
    }
  }
  if (union_fail) set_error(m, JZT_ERR_TIMEOUT, kStageFof);
  if (lane == 0 && pairs) atomicAdd(&m->fof_pairs, pairs);
}

// Canonical labels: point roots after the final contraction (a root starts its
// group's minimum original index with its own; only roots' entries of minorig
// are ever read), the members' minimum, then the labels in input order.
__global__ void k_contract_points(int32_t* ig_pt, const float4* __restrict__ pts, int32_t* minorig, int64_t n,
                                  const Meta* m) {
  if (failed(m)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = uf_root_ro(ig_pt, (int)i);
    ig_pt[i] = r;
    if (r == (int)i) minorig[i] = __float_as_int(pts[i].w);
  }
}

// The other members lower their root's minimum (singletons, most points at small
// linking lengths, need no atomic).
__global__ void k_group_min(const float4* __restrict__ pts, const int32_t* __restrict__ ig_pt,
                            int32_t* minorig, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = ig_pt[i];
    if (r != (int)i) atomicMin(&minorig[r], __float_as_int(pts[i].w));
  }
}

__global__ void k_labels(const float4* __restrict__ pts, const int32_t* __restrict__ ig_pt,
                         const int32_t* __restrict__ minorig, int32_t* labels, int64_t n,
                         const Meta* m) {
  if (failed(m)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    labels[__float_as_int(pts[i].w)] = minorig[ig_pt[i]];
}

int grid_for(int64_t work, int threads, int max_blocks) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

template <bool PER>
void fof_all(const Layout& L, char* ws, float pl, float b, int32_t* labels, cudaStream_t s) {
  Meta* m = at<Meta>(ws, L.meta);
  const int sms = 152;
  const int P = L.n_planes;
  const int64_t n = L.n;
  const float b2 = b * b;  // float32, round to nearest
  int2* arena = at<int2>(ws, L.arena);
  const int64_t cap = L.cap_ilist;  // IEntry and int2 are both 8 bytes
  prof_begin(kPhFofTop, s);
  k_fof_reset<<<1, 32, 0, s>>>(m); note_launch();
  launch_super_level(L, ws, s);
  k_fof_super_pairs<<<grid_for(L.cap_nodes[P], 128, sms * 4), 128, 0, s>>>(arena, P, cap,
                                                                            (int64_t)L.total, m); note_launch();
  k_fof_init_top<<<grid_for(L.cap_nodes[P - 1], 256, sms * 8), 256, 0, s>>>(
      at<NodeRec>(ws, L.nodes[P - 1]), at<int32_t>(ws, L.ig[P - 1]), at<uint8_t>(ws, L.lk[P - 1]),
      P - 1, pl, b2, m); note_launch();
  prof_end(kPhFofTop, s);
  for (int p = P - 1; p >= 0; --p) {
    prof_begin(kPhFofN2N, s);
    k_mark_plane_start<<<1, 32, 0, s>>>(m, p); note_launch();
    k_n2n_fof<PER><<<grid_for(L.cap_nodes[p + 1] * 32, 32 * kFofWarps, sms * 16), 32 * kFofWarps, 0, s>>>(
        at<int32_t>(ws, L.spl[p + 1]), at<NodeRec>(ws, L.nodes[p]), at<int32_t>(ws, L.ig[p]),
        at<uint8_t>(ws, L.lk[p]), arena, p + 1, pl, b2, cap, (int64_t)L.total, m); note_launch();
    k_mark_plane_end<<<1, 32, 0, s>>>(m, p); note_launch();
    k_contract<<<grid_for(L.cap_nodes[p], 256, sms * 8), 256, 0, s>>>(at<int32_t>(ws, L.ig[p]), p, 0, m); note_launch();
    if (p > 0) {
      k_parent_to_node<PER><<<grid_for(L.cap_nodes[p] * 32, 256, sms * 16), 256, 0, s>>>(
          at<int32_t>(ws, L.spl[p]), at<int32_t>(ws, L.ig[p]), at<uint8_t>(ws, L.lk[p]),
          at<NodeRec>(ws, L.nodes[p - 1]), at<int32_t>(ws, L.ig[p - 1]), at<uint8_t>(ws, L.lk[p - 1]),
          p, pl, b2, m); note_launch();
    }
    prof_end(kPhFofN2N, s);
  }
  int32_t* ig_pt = at<int32_t>(ws, L.ig_pt);
  prof_begin(kPhFofL2L, s);
  k_leaf_to_points<<<grid_for(L.cap_nodes[0] * 32, 256, sms * 16), 256, 0, s>>>(
      at<int32_t>(ws, L.spl[0]), at<int32_t>(ws, L.ig[0]), at<uint8_t>(ws, L.lk[0]), ig_pt, m); note_launch();
  k_l2l_fof<PER><<<sms * 16, 128, 0, s>>>(at<float4>(ws, L.pts), at<NodeRec>(ws, L.nodes[0]), arena,
                                          ig_pt, pl, b2, m); note_launch();
  prof_end(kPhFofL2L, s);
  prof_begin(kPhFofLabels, s);
  int32_t* minorig = at<int32_t>(ws, L.minorig);
  k_contract_points<<<grid_for(n, 256, sms * 8), 256, 0, s>>>(ig_pt, at<float4>(ws, L.pts), minorig, n, m);
  note_launch();
  k_group_min<<<grid_for(n, 256, sms * 8), 256, 0, s>>>(at<float4>(ws, L.pts), ig_pt, minorig, n); note_launch();
  k_labels<<<grid_for(n, 256, sms * 8), 256, 0, s>>>(at<float4>(ws, L.pts), ig_pt, minorig, labels, n, m); note_launch();
  prof_end(kPhFofLabels, s);
}

}  // namespace

void launch_fof(const Layout& L, char* ws, float periodic_L, float b, int32_t* d_labels,
                cudaStream_t s) {
  if (periodic_L > 0.0f) fof_all<true>(L, ws, periodic_L, b, d_labels, s);
  else fof_all<false>(L, ws, 0.0f, b, d_labels, s);
}

}  // namespace jzt
