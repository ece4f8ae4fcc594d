// Tree construction on the device (Sec. II): domain, Morton keys, the key sort
// (fine-bin bucket sort, or LSD radix passes), gather, gap levels and
// tree-plane splits, node records.
//
// Layout in HBM (all in the caller's workspace):
//   keys  uint64[N] x2 and vals uint32[N] x2 (radix ping-pong), sorted points
//   float4[N] (x, y, z, original index bits), per plane: splits int32[n+1],
//   point-space gap index int32[n+1], node size at each split int32[n+1] and
//   32-byte node records.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "zorder.cuh"

namespace jzt {

namespace {


__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inclusive scan within a warp.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan over a block of NT threads (one value each); returns the
// exclusive prefix and writes the block total to *total.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t s_w[NT / 32];
  __shared__ uint32_t s_tot;
  uint32_t inc = warp_incl_scan(v);
  if (lane_id() == 31) s_w[warp_id()] = inc;
  __syncthreads();
  if (warp_id() == 0) {
    uint32_t w = lane_id() < NT / 32 ? s_w[lane_id()] : 0u;
    uint32_t wi = warp_incl_scan(w);
    if (lane_id() < NT / 32) s_w[lane_id()] = wi - w;
    if (lane_id() == 31) s_tot = wi;  // lanes past NT/32 add zero: lane 31 holds the total
  }
  __syncthreads();
  uint32_t res = s_w[warp_id()] + inc - v;
  *total = s_tot;
  __syncthreads();  // s_w / s_tot may be reused by the caller's next scan
  return res;
}

// Decoupled look-back over tiles with one counter per tile (single-pass chained
// scan).  Called by one full warp; returns the exclusive prefix of `count` over
// tiles 0..tile-1 in every lane and publishes this tile's inclusive prefix.
// Waits are bounded: on exhaustion the status is set to JZT_ERR_TIMEOUT.
__device__ unsigned long long chained_scan(unsigned long long* st, int64_t tile, uint32_t count,
                                           Meta* m, int stage) {
  const unsigned long long A = 1ull << 62, P = 2ull << 62, MASK = (1ull << 62) - 1;
  const int lane = lane_id();
  if (tile == 0) {
    if (lane == 0) st_release_u64(&st[0], P | count);
    return 0;
  }
  if (lane == 0) st_release_u64(&st[tile], A | count);
  unsigned long long excl = 0;
  int64_t j = tile - 1;
  long long spins = 0;
  while (true) {
    int64_t t = j - lane;
    unsigned long long v = (t >= 0) ? ld_acquire_u64(&st[t]) : P;
    unsigned flag = (unsigned)(v >> 62);
    unsigned pm = __ballot_sync(0xffffffffu, flag == 2);
    unsigned nr = __ballot_sync(0xffffffffu, flag == 0);
    unsigned long long need = pm ? (((unsigned long long)(pm & (0u - pm)) << 1) - 1ull) : 0xffffffffull;
    if (nr & (unsigned)need) {
      if (++spins > kSpinLimit || failed(m)) {
        if (lane == 0) set_error(m, JZT_ERR_TIMEOUT, stage);
        break;
      }
      continue;
    }
    unsigned long long val = ((need >> lane) & 1ull) ? (v & MASK) : 0ull;
    excl += warp_sum(val);
    if (pm) break;
    j -= 32;
  }
  if (lane == 0) st_release_u64(&st[tile], P | (excl + count));
  return excl;
}

// ------------------------------------------------------------------ meta / box

__global__ void k_init_meta(Meta* m, int n_planes, int bucket_sort) {
  int t = threadIdx.x;
  if (t == 0) {
    m->status = 0;
    m->detail = 0;
    m->required_bytes = 0;
    m->arena_used = 0;
    m->arena_peak = 0;
    m->n_planes = n_planes;
  }
  if (t < 3) {
    m->bbox_enc[t] = 0xffffffffu;
    m->bbox_enc[3 + t] = 0u;
  }
  if (t < kMaxPlanes + 1) {
    m->n_nodes[t] = 0;
    m->pair_off[t] = 0;
    m->pair_cnt[t] = 0;
  }
  if (t < kMaxPlanes) {
    m->knn_plane_entries[t] = 0;
    m->reg_lvl[t] = kNoRegLevel;
  }
  if (t < kVolBins) m->vol_hist[t] = 0;
  if (t < 8) m->knn_stats[t] = 0;
  if (t == 0) {
    m->knn_pairs = 0;
    m->fof_pairs = 0;
    m->bucket_max = bucket_sort ? 0u : 0xffffffffu;  // no bucket sort tried: as if rejected
    m->big_bins = 0;
    m->big_next = 0;
  }
  if (t < 32) m->tile_ctr[t] = 0;
  uint32_t* h = &m->radix_hist[0][0];
  for (int i = t; i < kMaxRadixPasses * kMaxRadixBins; i += blockDim.x) h[i] = 0;
}

__global__ void k_zero_u64(unsigned long long* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0ull;
}

// The LSD radix passes of a build that tried the bucket sort run only when the
// device rejected it (a fine bin above kGrpStep keys); `gated` = 0: always.
__device__ __forceinline__ bool lsd_skipped(const Meta* m, int gated) {
  return gated && m->bucket_max <= (uint32_t)kGrpStep;
}

__global__ void k_zero_u64_gated(unsigned long long* p, int64_t n, const Meta* m) {
  if (lsd_skipped(m, 1)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0ull;
}

__device__ __forceinline__ bool bad_coord(float v, float L) {
  return !isfinite(v) || (L > 0.0f && (v < 0.0f || v >= L));
}

// Validation of every coordinate and, for open boxes, the bounding box
// (min/max reduction).  VEC: 16-byte aligned input read as float4 (3 float4 =
// 4 points).
template <bool VEC>
__global__ void __launch_bounds__(256) k_bbox(const float* __restrict__ xyz, int64_t n, float L,
                                              Meta* m) {
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  int64_t scalar_from = 0;
  if (VEC) {
    const int64_t ng = n / 4;
    const float4* p4 = reinterpret_cast<const float4*>(xyz);
    for (int64_t g = tid; g < ng; g += nth) {
      float4 a = __ldg(p4 + 3 * g), b = __ldg(p4 + 3 * g + 1), c = __ldg(p4 + 3 * g + 2);
      float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        const int d = e % 3;
        bad |= bad_coord(v[e], L);
        mn[d] = fminf(mn[d], v[e]);
        mx[d] = fmaxf(mx[d], v[e]);
      }
    }
    scalar_from = ng * 4;
  }
  for (int64_t i = scalar_from + tid; i < n; i += nth) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float v = xyz[3 * i + d];
      bad |= bad_coord(v, L);
      mn[d] = fminf(mn[d], v);
      mx[d] = fmaxf(mx[d], v);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) set_error(m, JZT_ERR_INPUT, kStageInput);
  if (L > 0.0f) return;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
      mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
    }
  }
  if (lane_id() == 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (mn[d] <= mx[d]) {
        atomicMin(&m->bbox_enc[d], f2sortable(mn[d]));
        atomicMax(&m->bbox_enc[3 + d], f2sortable(mx[d]));
      }
    }
  }
}

// Quantisation box: periodic -> origin 0, extent L; open -> origin at the
// minimum, common extent = the largest side (1 if all points coincide).
// scale = 2^21 / extent, rounded to nearest in float32.
__global__ void k_finish_box(Meta* m, float L) {
  if (threadIdx.x != 0) return;
  float ext;
  if (L > 0.0f) {
    m->lo[0] = m->lo[1] = m->lo[2] = 0.0f;
    ext = L;
  } else {
    ext = 0.0f;
    for (int d = 0; d < 3; ++d) {
      float lo = sortable2f(m->bbox_enc[d]);
      float hi = sortable2f(m->bbox_enc[3 + d]);
      m->lo[d] = lo;
      ext = fmaxf(ext, __fsub_rn(hi, lo));
    }
    if (!(ext > 0.0f)) ext = 1.0f;
  }
  m->scale = __fdiv_rn((float)(1 << kKeyBits), ext);
}

// ------------------------------------------------------------------ Morton keys

// Spread the low 21 bits of v so that bit j lands at bit 3j.
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint32_t quant(float v, float lo, float scale) {
  float u = __fmul_rn(__fsub_rn(v, lo), scale);
  uint32_t q = __float2uint_rd(u);
  return q > (1u << kKeyBits) - 1 ? (1u << kKeyBits) - 1 : q;
}

// Key bit 3j+2 = q_x bit j, 3j+1 = q_y bit j, 3j = q_z bit j (x most significant).
__device__ __forceinline__ uint64_t morton(float x, float y, float z, const float* lo, float sc) {
  return (spread3(quant(x, lo[0], sc)) << 2) | (spread3(quant(y, lo[1], sc)) << 1) |
         spread3(quant(z, lo[2], sc));
}

// Histogram of all radix digits of the keys held by a warp (lanes with
// valid=false contribute nothing).  A digit shared by the whole warp (the high
// digits of spatially coherent input) is added once; otherwise every lane adds
// its own (shared-memory atomics resolve the few collisions of random digits).
__device__ __forceinline__ void hist_key(uint32_t (*sh)[kRadixBins], uint64_t key, bool valid) {
  const unsigned act = __ballot_sync(0xffffffffu, valid);
  if (!valid) return;
  const int leader = __ffs(act) - 1;
#pragma unroll
  for (int p = 0; p < kRadixPasses; ++p) {
    uint32_t d = (uint32_t)(key >> (p * kRadixBits)) & (kRadixBins - 1);
    const uint32_t d0 = __shfl_sync(act, d, leader);
    if (__all_sync(act, d == d0)) {
      if (lane_id() == leader) atomicAdd(&sh[p][d], (uint32_t)__popc(act));
    } else {
      atomicAdd(&sh[p][d], 1u);
    }
  }
}

// Fine-bin counts of a thread's consecutive keys: one atomic per run of equal bins.
__device__ __forceinline__ void fine_count(uint32_t* __restrict__ fine, const uint64_t (&k4)[4], int cnt,
                                           int shift) {
  uint32_t bin = 0, run = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (e < cnt) {
      const uint32_t b = (uint32_t)(k4[e] >> shift);
      if (run && b == bin) {
        ++run;
      } else {
        if (run) atomicAdd(&fine[bin], run);
        bin = b;
        run = 1;
      }
    }
  }
  if (run) atomicAdd(&fine[bin], run);
}

// Keys of all points plus either the digit histograms of the LSD passes
// (fine == nullptr) or the counts of the 2^F fine bins (key >> fshift).  With
// check_L > 0 (periodic boxes, whose quantisation box needs no pass over the
// points) the coordinates are validated here instead of in k_bbox.
template <bool VEC>
__global__ void __launch_bounds__(256) k_keygen(const float* __restrict__ xyz, int64_t n, Meta* m,
                                                uint64_t* __restrict__ keys, uint32_t* __restrict__ fine,
                                                int fshift, float check_L) {
  bool bad = false;
  __shared__ uint32_t sh[kRadixPasses][kRadixBins];
  const bool digits = fine == nullptr;
  if (digits)
    for (int i = threadIdx.x; i < kRadixPasses * kRadixBins; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  const float lo[3] = {m->lo[0], m->lo[1], m->lo[2]};
  const float sc = m->scale;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t base_tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (VEC) {
    const int64_t ng = (n + 3) / 4;
    const int64_t ng_full = n / 4;
    const float4* p4 = reinterpret_cast<const float4*>(xyz);
    // iterate so that every lane of a warp runs the same number of rounds
    const int64_t rounds = (ng + nth - 1) / nth;
    for (int64_t r = 0; r < rounds; ++r) {
      int64_t g = r * nth + base_tid;
      uint64_t k4[4] = {0, 0, 0, 0};
      int cnt = 0;
      if (g < ng_full) {
        float4 a = __ldg(p4 + 3 * g), b = __ldg(p4 + 3 * g + 1), c = __ldg(p4 + 3 * g + 2);
        if (check_L > 0.0f) {
          const float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
          for (int e = 0; e < 12; ++e) bad |= bad_coord(v[e], check_L);
        }
        k4[0] = morton(a.x, a.y, a.z, lo, sc);
        k4[1] = morton(a.w, b.x, b.y, lo, sc);
        k4[2] = morton(b.z, b.w, c.x, lo, sc);
        k4[3] = morton(c.y, c.z, c.w, lo, sc);
        ulonglong2* o = reinterpret_cast<ulonglong2*>(keys + 4 * g);
        o[0] = make_ulonglong2(k4[0], k4[1]);
        o[1] = make_ulonglong2(k4[2], k4[3]);
        cnt = 4;
      } else if (g < ng) {
        cnt = (int)(n - 4 * g);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (e < cnt) {
            const int64_t i = 4 * g + e;
            if (check_L > 0.0f)
              bad |= bad_coord(xyz[3 * i], check_L) || bad_coord(xyz[3 * i + 1], check_L) ||
                     bad_coord(xyz[3 * i + 2], check_L);
            k4[e] = morton(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lo, sc);
            keys[i] = k4[e];
          }
        }
      }
      if (digits) {
#pragma unroll
        for (int e = 0; e < 4; ++e) hist_key(sh, k4[e], e < cnt);
      } else {
        fine_count(fine, k4, cnt, fshift);
      }
    }
  } else {
    const int64_t rounds = (n + nth - 1) / nth;
    for (int64_t r = 0; r < rounds; ++r) {
      int64_t i = r * nth + base_tid;
      uint64_t k = 0;
      if (i < n) {
        if (check_L > 0.0f)
          bad |= bad_coord(xyz[3 * i], check_L) || bad_coord(xyz[3 * i + 1], check_L) ||
                 bad_coord(xyz[3 * i + 2], check_L);
        k = morton(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lo, sc);
        keys[i] = k;
      }
      if (digits) hist_key(sh, k, i < n);
      else if (i < n) atomicAdd(&fine[k >> fshift], 1u);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) set_error(m, JZT_ERR_INPUT, kStageInput);
  if (!digits) return;
  __syncthreads();
  for (int i = threadIdx.x; i < kRadixPasses * kRadixBins; i += blockDim.x) {
    uint32_t v = (&sh[0][0])[i];
    if (v) atomicAdd(&m->radix_hist[i / kRadixBins][i % kRadixBins], v);
  }
}

// Exclusive digit offsets of `passes` passes of `bins` digits (one warp per pass).
__global__ void k_radix_offsets(Meta* m, int passes, int bins, int gated) {
  const int p = warp_id();
  if (p >= passes || lsd_skipped(m, gated)) return;
  uint32_t run = 0;
  for (int b0 = 0; b0 < bins; b0 += 32) {
    uint32_t v = m->radix_hist[p][b0 + lane_id()];
    uint32_t inc = warp_incl_scan(v);
    m->radix_offsets[p][b0 + lane_id()] = run + inc - v;
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
}

// ------------------------------------------------------------------ onesweep pass
//
// One stable counting pass of the LSD radix sort on the BITS-bit digit at bit
// `shift`.  Tiles of kSortTile keys are claimed in order through an atomic
// counter, so a tile only ever waits (decoupled look-back) on tiles that are
// already running.  A tile
//  1. loads kSortIpt keys per thread (striped over the warp: coalesced);
//  2. ranks every key among the keys of its warp with the same digit: the lanes
//     holding that digit are found with one ballot per digit bit, and the
//     lowest of them advances the warp's counter for the digit in shared memory;
//  3. per digit: prefix over the warps, tile count, tile start (block scan); the
//     tile counts are published for the later tiles at once;
//  4. moves its keys into shared memory in digit order -- which needs nothing
//     from other tiles -- and only then looks back for its global offsets, so
//     the tiles before it have had that much longer to publish;
//  5. writes its runs of equal digits, each contiguous in global memory.
// GATHER (the last pass of the build) writes, instead of the permutation, the
// sorted points float4(x, y, z, original index) read from the input by index.
//
// Look-back words (32 bit): 0 = nothing yet; kLbAgg | count = this tile's own
// count; otherwise 1 + the inclusive prefix over tiles 0..t (at most 2^31).
template <int BITS>
struct SortSmem {
  static constexpr int kBins = 1 << BITS;
  uint16_t whist[kSortThreads / 32][kBins];  // per-warp digit counts, then prefixes over warps
  uint32_t tile_start[kBins];
  uint32_t gbase[kBins];
  uint32_t tile;
  uint64_t stage_k[kSortTile];
  uint32_t stage_v[kSortTile];
};

constexpr uint32_t kLbAgg = 0xC0000000u;
constexpr int kLookWin = 8;  // predecessor words read per look-back step

// Exclusive prefix of digit d over the tiles before `tile`: walk back over the
// predecessors' words kLookWin at a time (independent relaxed loads: each word
// carries its own flag and value), adding tile counts until an inclusive prefix
// is found.  A word not yet published is polled again (bounded, with a short
// sleep); on exhaustion the status becomes JZT_ERR_TIMEOUT.
__device__ __forceinline__ uint32_t lookback_excl(const uint32_t* lookback, int64_t tile, int d, int bins,
                                                  Meta* m) {
  uint32_t excl = 0;
  int64_t j = tile - 1;
  long long spins = 0;
  while (j >= 0) {
    uint32_t v[kLookWin];
#pragma unroll
    for (int i = 0; i < kLookWin; ++i)
      v[i] = j - i >= 0 ? ld_relaxed_u32(lookback + (size_t)(j - i) * bins + d) : 1u;  // 1u: prefix 0
    int used = 0;
    bool found = false, blocked = false;
#pragma unroll
    for (int i = 0; i < kLookWin; ++i) {
      if (found || blocked) continue;
      if (v[i] == 0u) {
        blocked = true;
      } else if ((v[i] & kLbAgg) == kLbAgg) {
        excl += v[i] & ~kLbAgg;
        ++used;
      } else {
        excl += v[i] - 1u;
        found = true;
      }
    }
    if (found) break;
    j -= used;
    if (blocked) {
      if (++spins > kSpinLimit) {
        set_error(m, JZT_ERR_TIMEOUT, kStageSort);
        break;
      }
      if (failed(m)) break;
      __nanosleep(32);
    }
  }
  return excl;
}

template <int BITS, bool GATHER>
__global__ void __launch_bounds__(kSortThreads, 3)
    k_onesweep(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
               uint32_t* __restrict__ vout, int64_t n, int pass, int shift, uint32_t* lookback, Meta* m,
               const float* __restrict__ xa, const float* __restrict__ xb, int64_t na, float4* __restrict__ pts,
               int gated) {
  if (lsd_skipped(m, gated)) return;
  constexpr int kBins = 1 << BITS;
  constexpr int DPT = kBins / kSortThreads;  // digits per thread
  constexpr int W = kSortThreads / 32;
  static_assert(DPT >= 1 && DPT * kSortThreads == kBins, "whole digits per thread");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem<BITS>& S = *reinterpret_cast<SortSmem<BITS>*>(smem_raw);
  const int w = warp_id(), lane = lane_id(), t = threadIdx.x;
  if (t == 0) S.tile = atomicAdd(&m->tile_ctr[pass], 1u);
  for (int i = t; i < W * kBins; i += kSortThreads) (&S.whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = S.tile;
  const int64_t base = tile * kSortTile;
  const int tile_n = (int)min64(kSortTile, n - base);

  uint64_t key[kSortIpt];
  uint32_t val[kSortIpt];
  uint32_t rank[kSortIpt];
  uint32_t dig[kSortIpt];
  // key i of this thread sits at tile offset lofs + 32 i (striped over the warp)
  const int lofs = w * (32 * kSortIpt) + lane;
  const uint64_t* __restrict__ kp = kin + base + lofs;
  const uint32_t* __restrict__ vp = vin ? vin + base + lofs : nullptr;
#pragma unroll
  for (int i = 0; i < kSortIpt; ++i) {
    const bool ok = lofs + i * 32 < tile_n;
    key[i] = ok ? kp[i * 32] : 0ull;
    val[i] = ok ? (vp ? vp[i * 32] : (uint32_t)(base + lofs + i * 32)) : 0u;
    dig[i] = (uint32_t)(key[i] >> shift) & (kBins - 1);
  }
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kSortIpt; ++i) {
    const bool valid = lofs + i * 32 < tile_n;
    const uint32_t d = dig[i];
    unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
      const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
      peers &= ((d >> b) & 1u) ? bb : ~bb;
    }
    const int leader = valid ? __ffs(peers) - 1 : lane;
    uint32_t old = 0;
    if (valid && lane == leader) {
      old = S.whist[w][d];
      S.whist[w][d] = (uint16_t)(old + __popc(peers));
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rank[i] = old + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();
  // per digit (thread t owns digits t*DPT .. t*DPT+DPT-1): prefixes over warps and
  // the tile count, then the tile start of each digit (block scan)
  uint32_t cnt[DPT];
  uint32_t tsum = 0;
#pragma unroll
  for (int e = 0; e < DPT; ++e) {
    const int d = t * DPT + e;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < W; ++ww) {
      const uint32_t v = S.whist[ww][d];
      S.whist[ww][d] = (uint16_t)run;
      run += v;
    }
    cnt[e] = run;
    tsum += run;
  }
  uint32_t total;
  uint32_t start = block_excl_scan<kSortThreads>(tsum, &total);
  uint32_t* lb = lookback + (size_t)tile * kBins;
#pragma unroll
  for (int e = 0; e < DPT; ++e) {
    const int d = t * DPT + e;
    S.tile_start[d] = start;
    start += cnt[e];
    // tile 0 publishes its inclusive prefix (its count) directly
    st_relaxed_u32(&lb[d], tile == 0 ? cnt[e] + 1u : (kLbAgg | cnt[e]));
  }
  __syncthreads();
  // keys into shared memory in digit order
#pragma unroll
  for (int i = 0; i < kSortIpt; ++i) {
    if (lofs + i * 32 < tile_n) {
      const uint32_t d = dig[i];
      const uint32_t pos = S.tile_start[d] + S.whist[w][d] + rank[i];
      S.stage_k[pos] = key[i];
      S.stage_v[pos] = val[i];
    }
  }
  // global offset of every digit of this tile: look back over the tiles before it
#pragma unroll
  for (int e = 0; e < DPT; ++e) {
    const int d = t * DPT + e;
    uint32_t excl = 0;
    if (tile > 0) {
      excl = lookback_excl(lookback, tile, d, kBins, m);
      st_relaxed_u32(&lb[d], excl + cnt[e] + 1u);
    }
    S.gbase[d] = m->radix_offsets[pass][d] + excl;
  }
  __syncthreads();
  for (int j = t; j < tile_n; j += kSortThreads) {
    const uint64_t k = S.stage_k[j];
    const uint32_t d = (uint32_t)(k >> shift) & (kBins - 1);
    const uint32_t g = S.gbase[d] + (uint32_t)j - S.tile_start[d];
    if (g < (uint64_t)n) {  // always true unless a look-back wait gave up
      kout[g] = k;
      const uint32_t v = S.stage_v[j];
      if (GATHER) {
        const uint32_t p = v < (uint64_t)n ? v : 0u;
        const float* src = (int64_t)p < na ? xa + 3 * (int64_t)p : xb + 3 * ((int64_t)p - na);
        pts[g] = make_float4(__ldg(src), __ldg(src + 1), __ldg(src + 2), __uint_as_float(p));
      } else {
        vout[g] = v;
      }
    }
  }
}

// ---------------------------------------------------------------- bucket sort
//
// The same stable order of the integer keys (ties by original index) in fewer
// sweeps over memory and far fewer instructions per key, for sets whose fine
// bins (the top F key bits, about 32-64 keys each on average) each hold at most
// kGrpStep keys -- every nearly uniform set, the Zel'dovich lattices included:
//  1. k_keygen counts the keys per fine bin;
//  2. k_fine_scan turns the counts into each bin's first position (chained scan)
//     and records the largest count, which decides the path on the device;
//  3. k_bucket_scatter moves every (key, index) to its bin (order within a bin
//     arbitrary: one atomic per run of a warp's consecutive keys that share a bin);
//  4. k_bin_sort sorts each bin of at most kBinWarpMax keys by one warp, in
//     registers, with a bitonic network on (key, index) -- which also restores
//     the input order among equal keys -- and writes the sorted keys and the
//     sorted points float4(x, y, z, original index); larger bins are listed;
//  5. k_big_bins sorts the listed bins in shared memory by stable counting
//     passes over the bits that vary within the bin (index passes first where
//     equal keys occur).
// When a bin holds more than kGrpStep keys, steps 3-5 return at once and the
// LSD radix passes (launched gated) sort the keys of step 1 instead.
static_assert(kRadixPasses % 2 == 0, "the keys of an even number of LSD passes start in keys_a");
constexpr int kBinWarpMax = 128;   // bins up to this size: one warp, keys in registers
constexpr int kScatterRounds = 8;  // rounds of 32 keys per warp and chunk of the scatter

// Exclusive prefix of the fine-bin counts in place (fine) and as the scatter
// cursors (cur); tiles of kFineScanTile bins claimed in order, chained scan.
__global__ void __launch_bounds__(256) k_fine_scan(uint32_t* __restrict__ fine, uint32_t* __restrict__ cur,
                                                   int64_t nb, unsigned long long* st, Meta* m) {
  __shared__ int64_t s_tile;
  __shared__ unsigned long long s_pre;
  __shared__ uint32_t s_max;
  const int t = threadIdx.x;
  if (t == 0) {
    s_tile = atomicAdd(&m->tile_ctr[kCtrFine], 1u);
    s_max = 0;
  }
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * kFineScanTile + (int64_t)t * 16;  // nb is a multiple of 16
  uint32_t v[16];
  uint32_t sum = 0, mx = 0;
  if (base < nb) {
    const uint4* p4 = reinterpret_cast<const uint4*>(fine + base);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 u = p4[q];
      v[4 * q] = u.x;
      v[4 * q + 1] = u.y;
      v[4 * q + 2] = u.z;
      v[4 * q + 3] = u.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = 0;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    sum += v[i];
    mx = max(mx, v[i]);
  }
  if (mx) atomicMax(&s_max, mx);
  uint32_t total;
  const uint32_t ex = block_excl_scan<256>(sum, &total);
  if (warp_id() == 0) {
    const unsigned long long pre = chained_scan(st, tile, total, m, kStageSort);
    if (lane_id() == 0) s_pre = pre;
  }
  __syncthreads();
  if (t == 0 && s_max) atomicMax(&m->bucket_max, s_max);
  if (base >= nb) return;
  uint32_t run = (uint32_t)s_pre + ex;
  uint4* f4 = reinterpret_cast<uint4*>(fine + base);
  uint4* c4 = reinterpret_cast<uint4*>(cur + base);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint4 o;
    o.x = run;
    run += v[4 * q];
    o.y = run;
    run += v[4 * q + 1];
    o.z = run;
    run += v[4 * q + 2];
    o.w = run;
    run += v[4 * q + 3];
    f4[q] = o;
    c4[q] = o;
  }
}

// Every key (and its index) to the next free slot of its fine bin.  A warp takes
// 32 kScatterRounds consecutive keys, 32 per round (lane l: key 32 r + l); the
// lanes of a run of equal bins within a round take consecutive slots from one
// atomic of the run's first lane, so that they write consecutive addresses.  The
// atomics of all rounds are issued before any store.
__global__ void __launch_bounds__(256) k_bucket_scatter(const uint64_t* __restrict__ keys, int64_t n, int fshift,
                                                        uint32_t* __restrict__ cur, uint64_t* __restrict__ kb,
                                                        uint32_t* __restrict__ vb, const Meta* m) {
  if (m->bucket_max > (uint32_t)kGrpStep) return;
  constexpr int R = kScatterRounds;
  const int lane = lane_id();
  const unsigned upto = (2u << lane) - 1u;  // lanes <= lane (all ones for lane 31)
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_chunks = (n + 32 * R - 1) / (32 * R);
  for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += nw) {
    const int64_t base = c * 32 * R;
    uint64_t k[R];
    uint32_t bn[R], pos[R];
    unsigned starts[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t j = base + 32 * r + lane;
      k[r] = j < n ? keys[j] : 0ull;
      bn[r] = j < n ? (uint32_t)(k[r] >> fshift) : 0xffffffffu;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const bool valid = base + 32 * r + lane < n;  // the valid lanes are a prefix
      const uint32_t prev = __shfl_up_sync(0xffffffffu, bn[r], 1);
      const bool start = valid && (lane == 0 || prev != bn[r]);
      starts[r] = __ballot_sync(0xffffffffu, start);
      const unsigned vmask = __ballot_sync(0xffffffffu, valid);
      const unsigned after = starts[r] & ~upto;
      const int end = after ? __ffs(after) - 1 : __popc(vmask);
      pos[r] = start ? atomicAdd(&cur[bn[r]], (uint32_t)(end - lane)) : 0u;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t j = base + 32 * r + lane;
      const int leader = 31 - __clz(starts[r] & upto);
      const uint32_t p = __shfl_sync(0xffffffffu, pos[r], leader < 0 ? 0 : leader) + (uint32_t)(lane - leader);
      if (j < n && p < (uint64_t)n) {  // always in range: the counts came from the same keys
        kb[p] = k[r];
        vb[p] = (uint32_t)j;
      }
    }
  }
}

// Sorted key and point at sorted position g.
__device__ __forceinline__ void put_sorted(int64_t g, uint64_t key, uint32_t p0, int64_t n, uint64_t* __restrict__ kout,
                                           const float* __restrict__ xa, const float* __restrict__ xb, int64_t na,
                                           float4* __restrict__ pts) {
  kout[g] = key;
  const uint32_t p = p0 < (uint64_t)n ? p0 : 0u;
  const float* sp = (int64_t)p < na ? xa + 3 * (int64_t)p : xb + 3 * ((int64_t)p - na);
  pts[g] = make_float4(__ldg(sp), __ldg(sp + 1), __ldg(sp + 2), __uint_as_float(p));
}

// Bitonic network over the 32 E elements of a warp (element i = 32 e + lane in
// register e of the lane), ascending by key and, with FULL, by index among equal
// keys.
template <int E, bool FULL>
__device__ __forceinline__ void warp_bitonic(uint64_t (&k)[E], uint32_t (&v)[E]) {
  const int lane = lane_id();
#pragma unroll
  for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
    for (int st = size >> 1; st > 0; st >>= 1) {
      if (st >= 32) {
        const int es = st / 32;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if ((e & es) == 0) {
            const int f = e | es;
            const bool up = ((32 * e + lane) & size) == 0;
            const bool gt = k[e] > k[f] || (FULL && k[e] == k[f] && v[e] > v[f]);
            if (gt == up) {
              const uint64_t tk = k[e];
              k[e] = k[f];
              k[f] = tk;
              const uint32_t tv = v[e];
              v[e] = v[f];
              v[f] = tv;
            }
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint64_t ok = __shfl_xor_sync(0xffffffffu, k[e], st);
          const uint32_t ov = __shfl_xor_sync(0xffffffffu, v[e], st);
          const bool up = ((32 * e + lane) & size) == 0;
          const bool lower = (lane & st) == 0;
          // the lower slot of an ascending pair keeps the smaller; strict tests on both
          // sides, so that equal keys (compared without the index) stay where they are
          const bool other_less = ok < k[e] || (FULL && ok == k[e] && ov < v[e]);
          const bool other_more = ok > k[e] || (FULL && ok == k[e] && ov > v[e]);
          if ((lower == up) ? other_less : other_more) {
            k[e] = ok;
            v[e] = ov;
          }
        }
      }
    }
  }
}

// One bin of cnt <= 32 E keys sorted by one warp in registers (pads: all ones,
// after every key of 63 bits).  The network compares keys only; where equal keys
// end up adjacent it runs again comparing (key, index), which puts them in input
// order.
template <int E>
__device__ __forceinline__ void bin_sort_warp(const uint64_t* __restrict__ kb, const uint32_t* __restrict__ vb,
                                              int64_t e0, int cnt, int64_t n, uint64_t* __restrict__ kout,
                                              const float* __restrict__ xa, const float* __restrict__ xb, int64_t na,
                                              float4* __restrict__ pts) {
  const int lane = lane_id();
  uint64_t k[E];
  uint32_t v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = 32 * e + lane;
    k[e] = i < cnt ? kb[e0 + i] : ~0ull;
    v[e] = i < cnt ? vb[e0 + i] : ~0u;
  }
  warp_bitonic<E, false>(k, v);
  bool tie = false;
#pragma unroll
  for (int e = 0; e < E; ++e) {  // element i + 1: the next lane, or lane 0 of the next register
    const uint64_t dn = __shfl_down_sync(0xffffffffu, k[e], 1);
    const uint64_t wrap = __shfl_sync(0xffffffffu, k[e + 1 < E ? e + 1 : e], 0);
    const uint64_t nx = lane < 31 ? dn : wrap;
    const int i = 32 * e + lane;
    tie = tie || (i + 1 < cnt && nx == k[e]);
  }
  if (__any_sync(0xffffffffu, tie)) warp_bitonic<E, true>(k, v);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = 32 * e + lane;
    if (i < cnt) put_sorted(e0 + i, k[e], v[e], n, kout, xa, xb, na, pts);
  }
}

// Warps take chunks of 32 consecutive bins; bins above kBinWarpMax keys go to
// the list `big` (count in Meta::big_bins) for k_big_bins.
__global__ void __launch_bounds__(256) k_bin_sort(const uint64_t* __restrict__ kb, const uint32_t* __restrict__ vb,
                                                  const uint32_t* __restrict__ off, int64_t nb, int64_t n,
                                                  uint64_t* __restrict__ kout, const float* __restrict__ xa,
                                                  const float* __restrict__ xb, int64_t na, float4* __restrict__ pts,
                                                  uint32_t* __restrict__ big, Meta* m) {
  if (m->bucket_max > (uint32_t)kGrpStep) return;
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_chunks = (nb + 31) / 32;
  for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += nw) {
    const int64_t b = 32 * c + lane;
    const int64_t lo = b < nb ? (int64_t)off[b] : n;
    const int64_t hi = b + 1 < nb ? (int64_t)off[b + 1] : n;
    const int my_cnt = (int)(hi - lo);
    unsigned todo = __ballot_sync(0xffffffffu, my_cnt > 0);
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t e0 = __shfl_sync(0xffffffffu, lo, j);
      const int cnt = __shfl_sync(0xffffffffu, my_cnt, j);
      if (cnt <= 32) {
        bin_sort_warp<1>(kb, vb, e0, cnt, n, kout, xa, xb, na, pts);
      } else if (cnt <= 64) {
        bin_sort_warp<2>(kb, vb, e0, cnt, n, kout, xa, xb, na, pts);
      } else if (cnt <= kBinWarpMax) {
        bin_sort_warp<4>(kb, vb, e0, cnt, n, kout, xa, xb, na, pts);
      } else if (lane == 0) {
        big[atomicAdd(&m->big_bins, 1u)] = (uint32_t)(32 * c + j);
      }
    }
  }
}

struct GrpSmem {
  uint64_t k[2][kGrpCap];  // keys (ping-pong)
  uint32_t v[2][kGrpCap];  // original indices
  uint16_t whist[kGrpThreads / 32][256];
  uint32_t dstart[256];
  unsigned long long kx;   // OR over the bin of key ^ first key: the varying bits
  uint32_t vx;             // the same for the indices
  uint32_t item;
};

// One stable counting pass of the cnt elements of buffer src into src ^ 1 by the
// 8-bit digit at bit sh of the key (IDX: of the index).  Warp w ranks elements
// [w, w + 1) * 32 ipt, round i the 32 elements from 32 (w ipt + i): the order of
// (warp, round, lane) is the element order, so the pass is stable.
template <bool IDX>
__device__ __forceinline__ void grp_pass(GrpSmem& S, int src, int cnt, int ipt, int sh) {
  const int t = threadIdx.x, w = warp_id(), lane = lane_id();
  for (int i = t; i < (kGrpThreads / 32) * 256; i += kGrpThreads) (&S.whist[0][0])[i] = 0;
  __syncthreads();
  const unsigned lt = lanemask_lt();
  const int lofs = w * ipt * 32 + lane;
  uint32_t dig[kGrpIpt], rank[kGrpIpt];
#pragma unroll
  for (int i = 0; i < kGrpIpt; ++i) {
    dig[i] = 0;
    rank[i] = 0;
    if (i < ipt) {
      const int e = lofs + 32 * i;
      const bool valid = e < cnt;
      uint32_t d = 0;
      if (valid) d = IDX ? (S.v[src][e] >> sh) & 255u : (uint32_t)(S.k[src][e] >> sh) & 255u;
      unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bb : ~bb;
      }
      const int leader = valid ? __ffs(peers) - 1 : lane;
      uint32_t old = 0;
      if (valid && lane == leader) {
        old = S.whist[w][d];
        S.whist[w][d] = (uint16_t)(old + __popc(peers));
      }
      old = __shfl_sync(0xffffffffu, old, leader);
      dig[i] = d;
      rank[i] = old + __popc(peers & lt);
      __syncwarp();
    }
  }
  __syncthreads();
  // digit t: each warp's offset within the digit, then the digit's start
  uint32_t run = 0;
#pragma unroll
  for (int ww = 0; ww < kGrpThreads / 32; ++ww) {
    const uint32_t c = S.whist[ww][t];
    S.whist[ww][t] = (uint16_t)run;
    run += c;
  }
  uint32_t total;
  S.dstart[t] = block_excl_scan<kGrpThreads>(run, &total);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kGrpIpt; ++i) {
    const int e = lofs + 32 * i;
    if (i < ipt && e < cnt) {
      const uint32_t pos = S.dstart[dig[i]] + S.whist[w][dig[i]] + rank[i];
      S.k[src ^ 1][pos] = S.k[src][e];
      S.v[src ^ 1][pos] = S.v[src][e];
    }
  }
  __syncthreads();
}

// The listed bins (more than kBinWarpMax keys, at most kGrpStep <= kGrpCap),
// one at a time per block, taken from a shared counter.
__global__ void __launch_bounds__(kGrpThreads, 2)
    k_big_bins(const uint64_t* __restrict__ kb, const uint32_t* __restrict__ vb, const uint32_t* __restrict__ off,
               const uint32_t* __restrict__ big, int64_t nb, int64_t n, uint64_t* __restrict__ kout,
               const float* __restrict__ xa, const float* __restrict__ xb, int64_t na, float4* __restrict__ pts,
               Meta* m) {
  if (m->bucket_max > (uint32_t)kGrpStep) return;
  extern __shared__ __align__(16) unsigned char grp_smem[];
  GrpSmem& S = *reinterpret_cast<GrpSmem*>(grp_smem);
  const int t = threadIdx.x;
  const uint32_t n_big = m->big_bins;
  while (true) {
    if (t == 0) {
      S.item = atomicAdd(&m->big_next, 1u);
      S.kx = 0;
      S.vx = 0;
    }
    __syncthreads();
    const uint32_t item = S.item;
    if (item >= n_big) return;
    const int64_t b = big[item];
    const int64_t e0 = off[b];
    const int cnt = (int)((b + 1 < nb ? (int64_t)off[b + 1] : n) - e0);
    if (cnt > kGrpCap) {  // cannot happen while every bin holds at most kGrpStep keys
      if (t == 0) set_error(m, JZT_ERR_INTERNAL, kStageSort);
      return;
    }
    const uint64_t kf = kb[e0];
    const uint32_t vf = vb[e0];
    unsigned long long kx = 0;
    uint32_t vx = 0;
    for (int j = t; j < cnt; j += kGrpThreads) {
      const uint64_t k = kb[e0 + j];
      const uint32_t v = vb[e0 + j];
      S.k[0][j] = k;
      S.v[0][j] = v;
      kx |= k ^ kf;
      vx |= v ^ vf;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kx |= __shfl_xor_sync(0xffffffffu, kx, o);
      vx |= __shfl_xor_sync(0xffffffffu, vx, o);
    }
    if (lane_id() == 0) {
      if (kx) atomicOr(&S.kx, kx);
      if (vx) atomicOr(&S.vx, vx);
    }
    __syncthreads();
    const int hb = S.kx ? 64 - __clzll((long long)S.kx) : 0;
    const int ipt = (cnt + kGrpThreads - 1) / kGrpThreads;
    int src = 0;
    for (int sh = 0; sh < hb; sh += 8) {
      grp_pass<false>(S, src, cnt, ipt, sh);
      src ^= 1;
    }
    // equal keys are now adjacent but in the arbitrary order of the scatter: if
    // there are any, the passes run again over the index first
    bool eq = false;
    for (int j = t; j + 1 < cnt; j += kGrpThreads) eq = eq || S.k[src][j] == S.k[src][j + 1];
    if (__syncthreads_or(eq)) {
      const int hbv = S.vx ? 32 - __clz((int)S.vx) : 0;
      for (int sh = 0; sh < hbv; sh += 8) {
        grp_pass<true>(S, src, cnt, ipt, sh);
        src ^= 1;
      }
      for (int sh = 0; sh < hb; sh += 8) {
        grp_pass<false>(S, src, cnt, ipt, sh);
        src ^= 1;
      }
    }
    for (int j = t; j < cnt; j += kGrpThreads) put_sorted(e0 + j, S.k[src][j], S.v[src][j], n, kout, xa, xb, na, pts);
    __syncthreads();  // the buffers and S.item are reused by the next bin
  }
}

// Digit histograms of the LSD passes from the keys (bucket sort rejected).
__global__ void __launch_bounds__(256) k_lsd_hist(const uint64_t* __restrict__ keys, int64_t n, Meta* m) {
  if (lsd_skipped(m, 1)) return;
  __shared__ uint32_t sh[kRadixPasses][kRadixBins];
  for (int i = threadIdx.x; i < kRadixPasses * kRadixBins; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t rounds = (n + nth - 1) / nth;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t i = r * nth + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    hist_key(sh, i < n ? keys[i] : 0ull, i < n);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kRadixPasses * kRadixBins; i += blockDim.x) {
    const uint32_t v = (&sh[0][0])[i];
    if (v) atomicAdd(&m->radix_hist[i / kRadixBins][i % kRadixBins], v);
  }
}

// ---------------------------------------------------------------- two point sets
// Sorted positions are split by type, stably: sources keep their z order in
// pts2[0, n_src), queries in pts2[n_src, n) (Sec. II-G).  src_pos[i] = number
// of sources before sorted position i (src_pos[n] = n_src).
constexpr int kTypeThreads = 256;
constexpr int kTypePer = kScanTile / kTypeThreads;

__global__ void __launch_bounds__(kTypeThreads) k_src_tile_counts(const float4* __restrict__ pts, int64_t n,
                                                                  int64_t n_src, int32_t* tile_cnt) {
  __shared__ int32_t red[kTypeThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int c = 0;
#pragma unroll
  for (int e = 0; e < kTypePer; ++e) {
    const int64_t i = base + e * kTypeThreads + threadIdx.x;
    if (i < n) c += (int64_t)__float_as_uint(pts[i].w) < n_src ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane_id() == 0) red[warp_id()] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kTypeThreads / 32; ++w) t += red[w];
    tile_cnt[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile counts in place (one block; tiles <= 2^20).
__global__ void __launch_bounds__(1024) k_scan_tile_counts(int32_t* tile_cnt, int64_t n_tiles) {
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < n_tiles; b += 1024) {
    const int64_t i = b + threadIdx.x;
    const uint32_t v = i < n_tiles ? (uint32_t)tile_cnt[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_excl_scan<1024>(v, &total);
    if (i < n_tiles) tile_cnt[i] = carry + (int32_t)ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += (int32_t)total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kTypeThreads) k_split_types(const float4* __restrict__ pts, int64_t n,
                                                              int64_t n_src, const int32_t* __restrict__ tile_off,
                                                              float4* __restrict__ pts2, int32_t* __restrict__ src_pos) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kTypePer;  // blocked items
  float4 v[kTypePer];
  int c = 0;
#pragma unroll
  for (int e = 0; e < kTypePer; ++e) {
    const int64_t i = base + e;
    v[e] = i < n ? pts[i] : make_float4(0.f, 0.f, 0.f, __uint_as_float(0xffffffffu));
    c += (i < n && (int64_t)__float_as_uint(v[e].w) < n_src) ? 1 : 0;
  }
  uint32_t total;
  int32_t r = tile_off[blockIdx.x] + (int32_t)block_excl_scan<kTypeThreads>((uint32_t)c, &total);
#pragma unroll
  for (int e = 0; e < kTypePer; ++e) {
    const int64_t i = base + e;
    if (i >= n) break;
    src_pos[i] = r;
    const int64_t orig = (int64_t)__float_as_uint(v[e].w);
    if (orig < n_src) {
      pts2[r] = v[e];
      ++r;
    } else {
      pts2[n_src + (i - r)] = make_float4(v[e].x, v[e].y, v[e].z, __uint_as_float((uint32_t)(orig - n_src)));
    }
  }
  if (base <= n - 1 && n - 1 < base + kTypePer) src_pos[n] = (int32_t)n_src;
}

// Leaves: (first, count) become the source range in pts2; qrange = query range
// in the query part pts2 + n_src.  Boxes stay those of all points (conservative
// for either type).
__global__ void k_leaf_types(NodeRec* __restrict__ leaves, const int32_t* __restrict__ src_pos,
                             uint2* __restrict__ qrange, const Meta* m) {
  if (warp_failed(m)) return;
  const int64_t nl = m->n_nodes[0];
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nl; l += (int64_t)gridDim.x * blockDim.x) {
    NodeRec r = leaves[l];
    const int32_t s0 = src_pos[r.first], s1 = src_pos[r.first + r.count];
    qrange[l] = make_uint2((uint32_t)(r.first - s0), (uint32_t)(r.count - (s1 - s0)));
    r.first = s0;
    r.count = s1 - s0;
    leaves[l] = r;
  }
}

// Upper nodes: count = sum of the children's (source) counts.
__global__ void k_upper_counts(const int32_t* __restrict__ spl, const NodeRec* __restrict__ child,
                               NodeRec* __restrict__ nodes, int plane, const Meta* m) {
  if (warp_failed(m)) return;
  const int64_t nn = m->n_nodes[plane];
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = lane_id();
  for (int64_t P = gw; P < nn; P += nw) {
    int c = 0;
    for (int64_t ch = spl[P] + lane; ch < spl[P + 1]; ch += 32) c += child[ch].count;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) nodes[P].count = c;
  }
}

// ------------------------------------------------------------------ gap levels

// Level between sorted positions a < b: bit length of the key XOR; for equal
// keys the positions act as 32 extra low key bits, giving -clz(a ^ b) < 0.
__device__ __forceinline__ int level_ext(uint64_t ka, uint64_t kb, int64_t a, int64_t b) {
  uint64_t x = ka ^ kb;
  return x ? 64 - __clzll((long long)x) : -__clz((int)((uint32_t)a ^ (uint32_t)b));
}

// Leaf splits of plane 0 (Sec. II-C): gap i (0 < i < N) is a split when the
// smallest node holding points i-1 and i has n_i > M = N_max^(0) points.  Such a
// node holds M+1 consecutive points j..j+M around the gap exactly when the
// level of the pair (j, j+M) does not exceed the gap's level, for some
// j in [i-M, i-1]; the test reads only the keys within M of the gap (the range
// search of Sec. II-C, step 2).  Gaps 0 and N are always splits.  The flags
// are compacted in one pass (chained scan) into spl0 = split gap indices.
constexpr int kSplitThreads = 256;

// The two sources of levels: integer Morton keys (levels -32..64 fit in int8)
// and the float z-order of the sorted points themselves (levels -479..388).
struct KeyLevels {
  using Elem = uint64_t;
  using Lvl = int8_t;
  static constexpr int kNone = 127;
  static constexpr int kTile = 2048;  // gaps per tile (large tiles: few chained-scan steps)
  __device__ static Elem load(const void* src, int64_t pos) { return static_cast<const uint64_t*>(src)[pos]; }
  __device__ static Elem pad() { return 0ull; }
  __device__ static int level(const Elem& a, const Elem& b, int64_t ia, int64_t ib) { return level_ext(a, b, ia, ib); }
};
struct FloatLevels {
  using Elem = float4;
  using Lvl = int16_t;
  static constexpr int kNone = kZNoLevel;
  static constexpr int kTile = 2048;  // 16-byte elements: the tile's points fit 48 KB of shared memory
  __device__ static Elem load(const void* src, int64_t pos) { return static_cast<const float4*>(src)[pos]; }
  __device__ static Elem pad() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static int level(const Elem& a, const Elem& b, int64_t ia, int64_t ib) { return zlevel(a, b, ia, ib); }
};

template <class Src>
__global__ void __launch_bounds__(kSplitThreads) k_leaf_splits(const void* __restrict__ src,
                                                               int64_t n, int M, int32_t* spl0,
                                                               int64_t cap, unsigned long long* st,
                                                               Meta* m) {
  using Elem = typename Src::Elem;
  using Lvl = typename Src::Lvl;
  constexpr int kLeafTile = Src::kTile;
  constexpr int kSplitPer = kLeafTile / kSplitThreads;  // gaps per thread
  __shared__ Elem s_key[kLeafTile + 2 * 32 + 1];
  __shared__ Lvl s_w[kLeafTile + 32];
  __shared__ Lvl s_pre[kLeafTile + 32];
  __shared__ uint32_t s_tile;
  const int reg_lvl = m->reg_lvl[0];
  if (threadIdx.x == 0) s_tile = atomicAdd(&m->tile_ctr[kCtrLeafSplits], 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t g0 = tile * kLeafTile;
  // keys at positions [g0 - M, g0 + T + M)
  const int64_t k0 = g0 - M;
  const int nk = kLeafTile + 2 * M;
  for (int t = threadIdx.x; t < nk; t += kSplitThreads) {
    int64_t pos = k0 + t;
    s_key[t] = (pos >= 0 && pos < n) ? Src::load(src, pos) : Src::pad();
  }
  __syncthreads();
  // window levels w_j = level(j, j+M) for j in [g0 - M, g0 + T)
  for (int t = threadIdx.x; t < kLeafTile + M; t += kSplitThreads) {
    int64_t j = k0 + t;
    int v = Src::kNone;
    if (j >= 0 && j + M < n) v = Src::level(s_key[t], s_key[t + M], j, j + M);
    s_w[t] = (Lvl)v;
  }
  __syncthreads();
  // sliding minimum of width M over s_w by doubling: after step j, slot u holds the
  // minimum of s_w[u .. u + 2^(j+1) - 1]; with 2^kd <= M < 2^(kd+1) the window
  // [u, u + M - 1] is the union of the ranges of length 2^kd at u and u + M - 2^kd
  const int nw = kLeafTile + M;
  int kd = 0;
  while ((2 << kd) <= M) ++kd;
  Lvl* cur_t = s_w;
  Lvl* nxt_t = s_pre;
  for (int j = 0; j < kd; ++j) {
    const int d = 1 << j;
    for (int t = threadIdx.x; t < nw; t += kSplitThreads)
      nxt_t[t] = (Lvl)min((int)cur_t[t], t + d < nw ? (int)cur_t[t + d] : (int)Src::kNone);
    __syncthreads();
    Lvl* tmp = cur_t;
    cur_t = nxt_t;
    nxt_t = tmp;
  }
  const int span = 1 << kd;
  uint32_t flags = 0;
  int cnt = 0;
#pragma unroll
  for (int r = 0; r < kSplitPer; ++r) {
    int64_t i = g0 + threadIdx.x * kSplitPer + r;
    bool f = false;
    if (i == 0 || i == n) {
      f = true;
    } else if (i < n) {
      int li = (int)(i - k0);  // s_key index of point i
      int g = Src::level(s_key[li - 1], s_key[li], i - 1, i);
      f = reg_lvl != kNoRegLevel && g > reg_lvl;  // regularisation (Sec. II-D)
      // windows j in [i - M, i - 1] (slots u .. u + M - 1, u = i - g0; slots of
      // invalid j hold kNone): split when the smallest window level is <= g
      const int u = (int)(i - g0);
      const int wmin = min((int)cur_t[u], (int)cur_t[u + M - span]);
      f = f || wmin <= g;
    }
    flags |= (uint32_t)f << r;
    cnt += f;
  }
  uint32_t total;
  uint32_t local = block_excl_scan<kSplitThreads>((uint32_t)cnt, &total);
  __shared__ unsigned long long s_base;
  if (warp_id() == 0) {
    unsigned long long ex = chained_scan(st, tile, total, m, kStageSplits);
    if (lane_id() == 0) s_base = ex;
  }
  __syncthreads();
  const unsigned long long base = s_base + local;
#pragma unroll
  for (int r = 0, o = 0; r < kSplitPer; ++r) {
    if (flags >> r & 1u) {
      int64_t i = g0 + threadIdx.x * kSplitPer + r;
      unsigned long long pos = base + o++;
      if (pos <= (unsigned long long)cap) {
        spl0[pos] = (int32_t)i;
      } else {
        set_error(m, JZT_ERR_CAPACITY, kStageSplits);
      }
      if (i == n) m->n_nodes[0] = (int32_t)minu64(pos, (unsigned long long)cap);
    }
  }
}

// n_i at every plane-0 split gap (Sec. II-C: binary searches left and right for
// l_b and r_b; galloping from the gap since most nodes are small).
__device__ __forceinline__ int64_t first_ge_left(const uint64_t* keys, int64_t hi, int64_t lo_lim,
                                                 uint64_t target) {
  // smallest j in [lo_lim, hi] with keys[j] >= target, given keys[hi] >= target
  int64_t good = hi, step = 1;
  while (good - step >= lo_lim && keys[good - step] >= target) {
    good -= step;
    step <<= 1;
  }
  int64_t bad = max64(lo_lim - 1, good - step);  // keys[bad] < target or bad < lo_lim
  while (good - bad > 1) {
    int64_t mid = bad + (good - bad) / 2;
    if (keys[mid] >= target) good = mid; else bad = mid;
  }
  return good;
}
__device__ __forceinline__ int64_t first_gt_right(const uint64_t* keys, int64_t lo, int64_t hi_lim,
                                                  uint64_t target) {
  // smallest j in [lo, hi_lim] with j == hi_lim or keys[j] > target, given keys[lo-1] <= target
  int64_t good = lo - 1, step = 1;
  while (good + step < hi_lim && keys[good + step] <= target) {
    good += step;
    step <<= 1;
  }
  int64_t bad = min64(hi_lim, good + step);
  while (bad - good > 1) {
    int64_t mid = good + (bad - good) / 2;
    if (keys[mid] <= target) good = mid; else bad = mid;
  }
  return bad;
}

__global__ void k_split_sizes(const uint64_t* __restrict__ keys, int64_t n,
                              const int32_t* __restrict__ spl0, int32_t* __restrict__ nsz,
                              const Meta* m) {
  if (failed(m)) return;
  const int64_t ns = (int64_t)m->n_nodes[0] + 1;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = spl0[s];
    int64_t sz = n;
    if (i > 0 && i < n) {
      uint64_t ka = keys[i - 1], kb = keys[i];
      int g = level_ext(ka, kb, i - 1, i);
      if (g > 0) {
        uint64_t mask = (g >= 64) ? ~0ull : ((1ull << g) - 1ull);
        uint64_t lo_key = kb & ~mask, hi_key = kb | mask;
        int64_t lb = first_ge_left(keys, i - 1, 0, lo_key);
        int64_t rb = first_gt_right(keys, i + 1, n, hi_key);
        sz = rb - lb;
      } else {
        int bits = g + kIndexLevelOffset;
        int64_t blk = (i >> bits) << bits;
        int64_t blk_end = min64(n, blk + (1ll << bits));
        int64_t lb = first_ge_left(keys, i - 1, blk, kb);        // equal keys: keys[j] >= kb
        int64_t rb = first_gt_right(keys, i + 1, blk_end, kb);   // keys[j] > kb
        sz = rb - lb;
      }
    }
    nsz[s] = (int32_t)sz;
  }
}

// ---------------------------------------------------------------- float z-order (Sec. II-A)
// The full-precision alternative to the 21-bit keys: the points are sorted by the
// comparator of Eq. msb (zorder.cuh) with their original indices as the last key
// (a stable sort of the input), by a merge sort -- bitonic tiles of kFSortTile
// points in shared memory, then merge passes that split their output by merge
// path -- and the tree's levels come from the sorted points themselves.
constexpr int kFSortThreads = 256;
constexpr int kFSortTile = 2048;
constexpr int kFMergePer = 8;  // outputs per thread of a merge pass

// Pads (index >= n) sort after every point.
__device__ __forceinline__ bool fs_less(const float4& a, const float4& b, uint32_t n) {
  const uint32_t ia = __float_as_uint(a.w), ib = __float_as_uint(b.w);
  const bool pa = ia >= n, pb = ib >= n;
  if (pa != pb) return pb;
  if (pa) return ia < ib;
  return zless(a, b);
}

// Tile t of the combined index (p < na: xa[p], else xb[p - na]) sorted into out.
__global__ void __launch_bounds__(kFSortThreads) k_fsort_tiles(const float* __restrict__ xa,
                                                               const float* __restrict__ xb, int64_t na,
                                                               int64_t n, float4* __restrict__ out) {
  __shared__ float4 s[kFSortTile];
  const int64_t base = (int64_t)blockIdx.x * kFSortTile;
  for (int i = threadIdx.x; i < kFSortTile; i += kFSortThreads) {
    const int64_t p = base + i;
    if (p < n) {
      const float* src = p < na ? xa + 3 * p : xb + 3 * (p - na);
      s[i] = make_float4(src[0], src[1], src[2], __uint_as_float((uint32_t)p));
    } else {
      s[i] = make_float4(0.f, 0.f, 0.f, __uint_as_float((uint32_t)min64(p, 0xffffffffll)));
    }
  }
  __syncthreads();
  const uint32_t nn = (uint32_t)n;
  for (int size = 2; size <= kFSortTile; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = threadIdx.x; q < kFSortTile / 2; q += kFSortThreads) {
        const int i = 2 * q - (q & (stride - 1));
        const int j = i + stride;
        const bool up = (i & size) == 0;
        const float4 a = s[i], b = s[j];
        if (up ? fs_less(b, a, nn) : fs_less(a, b, nn)) {
          s[i] = b;
          s[j] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < kFSortTile; i += kFSortThreads)
    if (base + i < n) out[base + i] = s[i];
}

// One merge pass: runs [2wk, 2wk + w) and [2wk + w, 2wk + 2w) of in are merged
// into out.  Each thread writes kFMergePer consecutive outputs; the number of
// them taken from the first run is found by binary search on the merge path.
__global__ void __launch_bounds__(256) k_fsort_merge(const float4* __restrict__ in, float4* __restrict__ out,
                                                     int64_t n, int64_t w) {
  const int64_t o0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kFMergePer;
  if (o0 >= n) return;
  const uint32_t nn = (uint32_t)n;
  const int64_t base = (o0 / (2 * w)) * (2 * w);
  const int64_t la = min64(w, n - base);
  const int64_t lb = max64(0, min64(w, n - base - w));
  const float4* A = in + base;
  const float4* B = in + base + la;
  const int64_t d = o0 - base;
  int64_t lo = max64(0, d - lb), hi = min64(d, la);
  while (lo < hi) {  // a = how many of the first d outputs come from A
    const int64_t mid = (lo + hi) >> 1;
    if (fs_less(B[d - 1 - mid], A[mid], nn)) hi = mid;
    else lo = mid + 1;
  }
  int64_t ia = lo, ib = d - lo;
  const int64_t end = min64(o0 + kFMergePer, base + la + lb);
  for (int64_t o = o0; o < end; ++o) {
    const bool take_a = ia < la && (ib >= lb || !fs_less(B[ib], A[ia], nn));
    out[o] = take_a ? A[ia++] : B[ib++];
  }
}

// Predicate-driven forms of the galloping searches of k_split_sizes.
// Smallest j in [lo_lim, hi] such that in(j'') holds for all j'' in [j, hi], given in(hi).
template <class Pred>
__device__ __forceinline__ int64_t gallop_left(int64_t hi, int64_t lo_lim, Pred in) {
  int64_t good = hi, step = 1;
  while (good - step >= lo_lim && in(good - step)) {
    good -= step;
    step <<= 1;
  }
  int64_t bad = max64(lo_lim - 1, good - step);
  while (good - bad > 1) {
    const int64_t mid = bad + (good - bad) / 2;
    if (in(mid)) good = mid; else bad = mid;
  }
  return good;
}
// Smallest j in [lo, hi_lim] with j == hi_lim or !in(j), given in(lo - 1).
template <class Pred>
__device__ __forceinline__ int64_t gallop_right(int64_t lo, int64_t hi_lim, Pred in) {
  int64_t good = lo - 1, step = 1;
  while (good + step < hi_lim && in(good + step)) {
    good += step;
    step <<= 1;
  }
  int64_t bad = min64(hi_lim, good + step);
  while (bad - good > 1) {
    const int64_t mid = good + (bad - good) / 2;
    if (in(mid)) good = mid; else bad = mid;
  }
  return bad;
}

// n_i at every plane-0 split gap on the float order: the node at level lvl_i that
// holds points i-1 and i is the contiguous range of the points j with
// level(j, i) <= lvl_i (equal points: the equal points in the same aligned
// block of sorted positions).
__global__ void k_split_sizes_f(const float4* __restrict__ pts, int64_t n, const int32_t* __restrict__ spl0,
                                int32_t* __restrict__ nsz, const Meta* m) {
  if (failed(m)) return;
  const int64_t ns = (int64_t)m->n_nodes[0] + 1;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = spl0[s];
    int64_t sz = n;
    if (i > 0 && i < n) {
      const float4 pi = pts[i];
      const int g = zlevel(pts[i - 1], pi, i - 1, i);
      if (g > kZIndexLevel + 32) {
        auto in = [&](int64_t j) { return zlevel(pts[j], pi, j, i) <= g; };
        sz = gallop_right(i + 1, n, in) - gallop_left(i - 1, 0, in);
      } else {
        const int bits = g - kZIndexLevel;
        const int64_t blk = (i >> bits) << bits;
        const int64_t blk_end = min64(n, blk + (1ll << bits));
        auto same = [&](int64_t j) {
          int mk;
          const float4 q = pts[j];
          (void)zdim(q.x, q.y, q.z, pi.x, pi.y, pi.z, &mk);
          return mk < 0;
        };
        sz = gallop_right(i + 1, blk_end, same) - gallop_left(i - 1, blk, same);
      }
    }
    nsz[s] = (int32_t)sz;
  }
}

// Plane p >= 1: keep the plane p-1 splits whose n exceeds N_max^(p) (plus the
// two ends); spl[p] holds their positions in plane p-1's split array, gap[p]
// and nsz[p] carry the point-space gap index and n along.
// ---------------------------------------------------------------- regularisation
// Points per node-volume class of plane p (nodes [gap[j], gap[j+1])): 0 for one
// point, else 1 + 32 + level of the node (the level of its first and last point,
// the largest gap level inside it).
__global__ void k_vol_hist(const uint64_t* __restrict__ keys, const int32_t* __restrict__ gap, int plane,
                           Meta* m) {
  __shared__ unsigned long long sh[kVolBins];
  for (int i = threadIdx.x; i < kVolBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int64_t nn = m->n_nodes[plane];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = gap[j], b = gap[j + 1];
    const int bin = b - a >= 2 ? 1 + 32 + level_ext(keys[a], keys[b - 1], a, b - 1) : 0;
    atomicAdd(&sh[bin], (unsigned long long)(b - a));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kVolBins; i += blockDim.x)
    if (sh[i]) atomicAdd(&m->vol_hist[i], sh[i]);
}

// lvl_max^(p): 2^lvl_max <= f_max V_90%, V_90% = point-weighted mean node volume
// over the smallest nodes holding 90 % of the points (whole volume classes from
// the smallest; of the class that reaches 90 % only the points still needed).
// float64 in this exact order, no fused operations.  Clears the histogram.
__global__ void k_reg_level(int plane, int64_t n, float f_max, Meta* m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double target = __dmul_rn(0.9, (double)n);
  double acc = 0.0;
  long long cum = 0;
  for (int b = 0; b < kVolBins; ++b) {
    const long long h = (long long)m->vol_hist[b];
    if (h == 0) continue;
    const double vol = b == 0 ? 0.0 : ldexp(1.0, b - 33);
    if ((double)(cum + h) >= target) {
      acc = __dadd_rn(acc, __dmul_rn(__dsub_rn(target, (double)cum), vol));
      break;
    }
    acc = __dadd_rn(acc, __dmul_rn((double)h, vol));
    cum += h;
  }
  const double v90 = __ddiv_rn(acc, target);
  const double x = __dmul_rn((double)f_max, v90);
  int e = 0;
  if (x > 0.0) {
    (void)frexp(x, &e);
    m->reg_lvl[plane] = e - 1;
  } else {
    m->reg_lvl[plane] = kNoRegLevel;
  }
  for (int b = 0; b < kVolBins; ++b) m->vol_hist[b] = 0;
}

__global__ void k_reset_ctr(Meta* m, int ctr) {
  if (threadIdx.x == 0) m->tile_ctr[ctr] = 0;
}

__global__ void __launch_bounds__(256) k_coarse_splits(const int32_t* __restrict__ gap_in,
                                                       const int32_t* __restrict__ nsz_in,
                                                       int plane_in, int64_t nmax, int32_t* spl,
                                                       int32_t* gap_out, int32_t* nsz_out,
                                                       int64_t cap, unsigned long long* st,
                                                       int ctr, const uint64_t* __restrict__ keys,
                                                       int64_t n, Meta* m) {
  constexpr int PER = kScanTile / 256;
  __shared__ uint32_t s_tile;
  const int reg_lvl = m->reg_lvl[plane_in + 1];
  if (threadIdx.x == 0) s_tile = atomicAdd(&m->tile_ctr[ctr], 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t nin = (int64_t)m->n_nodes[plane_in] + 1;  // splits of the finer plane
  const int64_t t0 = tile * kScanTile + threadIdx.x * PER;
  uint32_t flags = 0;
  int cnt = 0;
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    int64_t t = t0 + r;
    bool f = false;
    if (t < nin) {
      f = (t == 0) || (t == nin - 1) || ((int64_t)nsz_in[t] > nmax);
      if (!f && reg_lvl != kNoRegLevel) {  // regularisation (Sec. II-D)
        const int64_t g = gap_in[t];
        f = g > 0 && g < n && level_ext(keys[g - 1], keys[g], g - 1, g) > reg_lvl;
      }
    }
    flags |= (uint32_t)f << r;
    cnt += f;
  }
  uint32_t total;
  uint32_t local = block_excl_scan<256>((uint32_t)cnt, &total);
  __shared__ unsigned long long s_base;
  if (warp_id() == 0) {
    unsigned long long ex = chained_scan(st, tile, total, m, kStageSplits);
    if (lane_id() == 0) s_base = ex;
  }
  __syncthreads();
  const unsigned long long base = s_base + local;
#pragma unroll
  for (int r = 0, o = 0; r < PER; ++r) {
    if (flags >> r & 1u) {
      int64_t t = t0 + r;
      unsigned long long pos = base + o++;
      if (pos <= (unsigned long long)cap) {
        spl[pos] = (int32_t)t;
        gap_out[pos] = gap_in[t];
        nsz_out[pos] = nsz_in[t];
      } else {
        set_error(m, JZT_ERR_CAPACITY, kStageSplits);
      }
      if (t == nin - 1) m->n_nodes[plane_in + 1] = (int32_t)minu64(pos, (unsigned long long)cap);
    }
  }
}

// ------------------------------------------------------------------ node records
// Leaves: one warp per leaf reduces its points' bounding box.
__global__ void k_leaf_nodes(const float4* __restrict__ pts, const int32_t* __restrict__ spl0,
                             NodeRec* __restrict__ nodes, const Meta* m) {
  // one lane per leaf: a warp's 32 leaves are consecutive, so its lanes read
  // neighbouring stretches of the sorted points and write consecutive records
  if (warp_failed(m)) return;
  const int64_t nn = m->n_nodes[0];
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < nn; L += nt) {
    const int64_t s = spl0[L], e = spl0[L + 1];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = s; i < e; ++i) {
      const float4 p = pts[i];
      lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
      hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
    }
    NodeRec r;
    r.lo[0] = lo[0]; r.lo[1] = lo[1]; r.lo[2] = lo[2];
    r.hi[0] = hi[0]; r.hi[1] = hi[1]; r.hi[2] = hi[2];
    r.count = (int32_t)(e - s);
    r.first = (int32_t)s;
    nodes[L] = r;
  }
}

// Plane p >= 1: one warp per node reduces its children's records.
__global__ void k_upper_nodes(const int32_t* __restrict__ spl, const int32_t* __restrict__ gap,
                              const NodeRec* __restrict__ child, NodeRec* __restrict__ nodes,
                              int plane, const Meta* m) {
  if (warp_failed(m)) return;
  const int64_t nn = m->n_nodes[plane];
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = lane_id();
  for (int64_t P = gw; P < nn; P += nw) {
    int64_t s = spl[P], e = spl[P + 1];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t c = s + lane; c < e; c += 32) {
      NodeRec r = child[c];
      lo[0] = fminf(lo[0], r.lo[0]); lo[1] = fminf(lo[1], r.lo[1]); lo[2] = fminf(lo[2], r.lo[2]);
      hi[0] = fmaxf(hi[0], r.hi[0]); hi[1] = fmaxf(hi[1], r.hi[1]); hi[2] = fmaxf(hi[2], r.hi[2]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
        hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
      }
    }
    if (lane == 0) {
      NodeRec r;
      r.lo[0] = lo[0]; r.lo[1] = lo[1]; r.lo[2] = lo[2];
      r.hi[0] = hi[0]; r.hi[1] = hi[1]; r.hi[2] = hi[2];
      r.count = gap[P + 1] - gap[P];
      r.first = (int32_t)s;
      nodes[P] = r;
    }
  }
}

// Super nodes (Alg. 1): NGR consecutive top nodes per super node.
__global__ void k_super_splits(int32_t* spl_super, int top_plane, int ngr, int64_t cap, Meta* m) {
  const int64_t ntop = m->n_nodes[top_plane];
  const int64_t nsup = (ntop + ngr - 1) / ngr;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (nsup > cap) set_error(m, JZT_ERR_CAPACITY, kStageTop);
    m->n_nodes[top_plane + 1] = (int32_t)min64(nsup, cap);
  }
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s <= min64(nsup, cap);
       s += (int64_t)gridDim.x * blockDim.x)
    spl_super[s] = (int32_t)min64(s * ngr, ntop);
}

int grid_for(int64_t work, int threads, int max_blocks) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

}  // namespace

void launch_super_level(const Layout& L, char* ws, cudaStream_t s) {
  Meta* m = at<Meta>(ws, L.meta);
  const int P = L.n_planes;
  k_super_splits<<<grid_for(L.cap_nodes[P] + 1, 256, 1024), 256, 0, s>>>(
      at<int32_t>(ws, L.spl[P]), P - 1, L.ngr, L.cap_nodes[P], m); note_launch();
}

namespace {

void bbox_part(const float* d, int64_t n, float periodic_L, Meta* m, cudaStream_t s) {
  const bool vec = (reinterpret_cast<uintptr_t>(d) & 15u) == 0;
  const int gb = grid_for((n + 3) / 4, 256, 152 * 8);
  if (vec) k_bbox<true><<<gb, 256, 0, s>>>(d, n, periodic_L, m);
  else k_bbox<false><<<gb, 256, 0, s>>>(d, n, periodic_L, m);
  note_launch();
}

void keygen_part(const float* d, int64_t n, Meta* m, uint64_t* keys, uint32_t* fine, int fshift,
                 float check_L, cudaStream_t s) {
  // the vectorised path loads float4 groups of points and stores key pairs as
  // 16-byte words: both addresses must be 16-byte aligned (the query part of a
  // two-set build starts at keys + n_src)
  const bool vec = (reinterpret_cast<uintptr_t>(d) & 15u) == 0 && (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
  const int gb = grid_for((n + 3) / 4, 256, 152 * 8);
  if (vec) k_keygen<true><<<gb, 256, 0, s>>>(d, n, m, keys, fine, fshift, check_L);
  else k_keygen<false><<<gb, 256, 0, s>>>(d, n, m, keys, fine, fshift, check_L);
  note_launch();
}

// Points a (n_a) then b (n_b; may be null with n_b = 0) under one combined index.
void build_impl(const float* d_a, int64_t n_a, const float* d_b, int64_t n_b, float periodic_L,
                const Layout& L, char* ws, cudaStream_t s) {
  const int64_t n = n_a + n_b;
  Meta* m = at<Meta>(ws, L.meta);
  const int sms = 152;
  prof_begin(kPhBox, s);
  k_init_meta<<<1, 256, 0, s>>>(m, L.n_planes, L.bucket_sort); note_launch();
  // periodic boxes with integer keys: the key generation validates the points
  const bool check_in_keys = !L.float_order && periodic_L > 0.0f;
  if (!check_in_keys) {
    bbox_part(d_a, n_a, periodic_L, m, s);
    if (n_b > 0) bbox_part(d_b, n_b, periodic_L, m, s);
  }
  k_finish_box<<<1, 32, 0, s>>>(m, periodic_L); note_launch();
  prof_end(kPhBox, s);
  uint64_t* keys_a = at<uint64_t>(ws, L.keys_a);
  float4* pts = at<float4>(ws, L.pts);
  if (L.float_order) {
    // float z-order (Sec. II-A): merge sort of the points by the comparator; the
    // passes alternate between pts and pts_tmp and end in pts
    prof_begin(kPhSort, s);
    float4* tmp = at<float4>(ws, L.pts_tmp);
    int merge_passes = 0;
    for (int64_t w = kFSortTile; w < n; w *= 2) ++merge_passes;
    float4* cur = (merge_passes % 2) ? tmp : pts;
    k_fsort_tiles<<<(unsigned)((n + kFSortTile - 1) / kFSortTile), kFSortThreads, 0, s>>>(d_a, d_b, n_a, n, cur);
    note_launch();
    for (int64_t w = kFSortTile; w < n; w *= 2) {
      float4* nxt = (cur == pts) ? tmp : pts;
      const int64_t threads = (n + kFMergePer - 1) / kFMergePer;
      k_fsort_merge<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(cur, nxt, n, w);
      note_launch();
      cur = nxt;
    }
    prof_end(kPhSort, s);
  } else {
  prof_begin(kPhKeys, s);
  uint64_t* keys_b = at<uint64_t>(ws, L.keys_b);
  uint32_t* vals_a = at<uint32_t>(ws, L.vals_a);
  uint32_t* vals_b = at<uint32_t>(ws, L.vals_b);
  // the passes alternate between the two key buffers and must end in keys_a:
  // with an odd number of passes the keys start in keys_b
  uint64_t* keys_in = (kRadixPasses % 2) ? keys_b : keys_a;
  uint32_t* lookback = at<uint32_t>(ws, L.lookback);
  // bucket sort: fine-bin counts, then first positions, and the scatter cursors
  // live in the look-back area, which the LSD passes need only when they run
  const int gated = L.bucket_sort ? 1 : 0;
  const int64_t nbins = (int64_t)1 << L.fine_bits;
  const int fshift = 3 * kKeyBits - L.fine_bits;
  uint32_t* fine = L.bucket_sort ? lookback : nullptr;
  uint32_t* fine_cur = lookback + nbins;
  uint32_t* big = lookback + 2 * nbins;  // bins for k_big_bins (at most n / (kBinWarpMax + 1))
  if (L.bucket_sort) {
    k_zero_u64<<<grid_for(nbins / 2, 256, sms * 8), 256, 0, s>>>(reinterpret_cast<unsigned long long*>(fine),
                                                                   nbins / 2);
    note_launch();
  }
  const float check_L = check_in_keys ? periodic_L : 0.0f;
  keygen_part(d_a, n_a, m, keys_in, fine, fshift, check_L, s);
  if (n_b > 0) keygen_part(d_b, n_b, m, keys_in + n_a, fine, fshift, check_L, s);
  if (L.bucket_sort) {
    unsigned long long* st = at<unsigned long long>(ws, L.scan_flags);
    const int64_t ft = (nbins + kFineScanTile - 1) / kFineScanTile;
    k_zero_u64<<<grid_for(ft, 256, sms * 8), 256, 0, s>>>(st, ft);
    k_fine_scan<<<(unsigned)ft, 256, 0, s>>>(fine, fine_cur, nbins, st, m);
    note_launch(2);
    prof_end(kPhKeys, s);
    prof_begin(kPhSort, s);
    k_bucket_scatter<<<grid_for((n + 31) / 32 * 32 / kScatterRounds, 256, sms * 8), 256, 0, s>>>(
        keys_in, n, fshift, fine_cur, keys_b, vals_b, m);
    k_bin_sort<<<grid_for((nbins + 31) / 32 * 32, 256, sms * 8), 256, 0, s>>>(keys_b, vals_b, fine, nbins, n, keys_a,
                                                                               d_a, d_b, n_a, pts, big, m);
    const size_t gsm = sizeof(GrpSmem);
    cudaFuncSetAttribute(k_big_bins, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    k_big_bins<<<sms * 2, kGrpThreads, gsm, s>>>(keys_b, vals_b, fine, big, nbins, n, keys_a, d_a, d_b, n_a, pts, m);
    note_launch(3);
    k_lsd_hist<<<grid_for((n + 3) / 4, 256, sms * 8), 256, 0, s>>>(keys_in, n, m);
    note_launch();
  }
  k_radix_offsets<<<1, 32 * kRadixPasses, 0, s>>>(m, kRadixPasses, kRadixBins, gated); note_launch();
  // look-back tables of all passes, zeroed once
  const int64_t lb_words = L.n_tiles_sort * kRadixBins * kRadixPasses;
  k_zero_u64_gated<<<grid_for(lb_words / 2 + 1, 256, sms * 8), 256, 0, s>>>(
      reinterpret_cast<unsigned long long*>(lookback), (lb_words + 1) / 2, m); note_launch();
  if (!L.bucket_sort) {
    prof_end(kPhKeys, s);
    prof_begin(kPhSort, s);
  }
  const size_t smem = sizeof(SortSmem<kRadixBits>);
  cudaFuncSetAttribute(k_onesweep<kRadixBits, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_onesweep<kRadixBits, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const uint64_t* kin = keys_in;
  const uint32_t* vin = nullptr;
  uint32_t* vout = vals_a;
  for (int p = 0; p < kRadixPasses; ++p) {
    uint64_t* kout = (kin == keys_a) ? keys_b : keys_a;
    uint32_t* lb = lookback + (size_t)p * L.n_tiles_sort * kRadixBins;
    if (p + 1 < kRadixPasses) {
      k_onesweep<kRadixBits, false><<<(unsigned)L.n_tiles_sort, kSortThreads, smem, s>>>(
          kin, vin, kout, vout, n, p, p * kRadixBits, lb, m, nullptr, nullptr, 0, nullptr, gated);
    } else {  // last pass: the sorted points (gather) instead of the permutation
      k_onesweep<kRadixBits, true><<<(unsigned)L.n_tiles_sort, kSortThreads, smem, s>>>(
          kin, vin, kout, nullptr, n, p, p * kRadixBits, lb, m, d_a, d_b, n_a, pts, gated);
    }
    note_launch();
    kin = kout;
    vin = vout;
    vout = (vout == vals_a) ? vals_b : vals_a;
  }
  prof_end(kPhSort, s);
  }  // integer keys
  prof_begin(kPhSplits, s);
  // plane 0: leaf splits, then n_i at every leaf split
  unsigned long long* st = at<unsigned long long>(ws, L.scan_flags);
  const int64_t leaf_tile = L.float_order ? FloatLevels::kTile : KeyLevels::kTile;
  const int64_t split_tiles = (n + 1 + leaf_tile - 1) / leaf_tile;
  const bool reg = L.reg_fmax > 0.0f;
  // regularisation (Sec. II-D): after a plane's count splits, the volume classes
  // of its nodes give lvl_max^(p); the plane's splits are then taken again with
  // the level criterion added
  auto regularise = [&](int p) {
    k_vol_hist<<<grid_for(L.cap_nodes[p], 256, sms * 8), 256, 0, s>>>(keys_a, at<int32_t>(ws, L.gap[p]), p, m);
    k_reg_level<<<1, 32, 0, s>>>(p, n, L.reg_fmax, m);
    k_reset_ctr<<<1, 32, 0, s>>>(m, p == 0 ? kCtrLeafSplits : kCtrCoarse + p);
    note_launch(3);
  };
  for (int pass = 0; pass < (reg ? 2 : 1); ++pass) {
    if (pass == 1) regularise(0);
    k_zero_u64<<<grid_for(split_tiles, 256, sms * 8), 256, 0, s>>>(st, split_tiles); note_launch();
    if (L.float_order) {
      k_leaf_splits<FloatLevels><<<(unsigned)split_tiles, kSplitThreads, 0, s>>>(
          pts, n, L.nmax0, at<int32_t>(ws, L.spl[0]), L.cap_nodes[0], st, m);
      k_split_sizes_f<<<grid_for(L.cap_nodes[0] + 1, 256, sms * 16), 256, 0, s>>>(
          pts, n, at<int32_t>(ws, L.spl[0]), at<int32_t>(ws, L.nsz[0]), m);
    } else {
      k_leaf_splits<KeyLevels><<<(unsigned)split_tiles, kSplitThreads, 0, s>>>(
          keys_a, n, L.nmax0, at<int32_t>(ws, L.spl[0]), L.cap_nodes[0], st, m);
      k_split_sizes<<<grid_for(L.cap_nodes[0] + 1, 256, sms * 16), 256, 0, s>>>(
          keys_a, n, at<int32_t>(ws, L.spl[0]), at<int32_t>(ws, L.nsz[0]), m);
    }
    note_launch(2);
  }
  // coarser planes
  int64_t nmax = L.nmax0;
  for (int p = 1; p < L.n_planes; ++p) {
    nmax *= L.c;
    const int64_t tiles = (L.cap_nodes[p - 1] + 1 + kScanTile - 1) / kScanTile;
    for (int pass = 0; pass < (reg ? 2 : 1); ++pass) {
      if (pass == 1) regularise(p);
      k_zero_u64<<<grid_for(tiles, 256, sms * 8), 256, 0, s>>>(st, tiles); note_launch();
      k_coarse_splits<<<(unsigned)tiles, 256, 0, s>>>(
          at<int32_t>(ws, L.gap[p - 1]), at<int32_t>(ws, L.nsz[p - 1]), p - 1, nmax,
          at<int32_t>(ws, L.spl[p]), at<int32_t>(ws, L.gap[p]), at<int32_t>(ws, L.nsz[p]),
          L.cap_nodes[p], st, kCtrCoarse + p, keys_a, n, m); note_launch();
    }
  }
  prof_end(kPhSplits, s);
  prof_begin(kPhNodes, s);
  // node records
  k_leaf_nodes<<<grid_for(L.cap_nodes[0], 256, sms * 16), 256, 0, s>>>(
      pts, at<int32_t>(ws, L.spl[0]), at<NodeRec>(ws, L.nodes[0]), m); note_launch();
  for (int p = 1; p < L.n_planes; ++p) {
    k_upper_nodes<<<grid_for(L.cap_nodes[p] * 32, 256, sms * 16), 256, 0, s>>>(
        at<int32_t>(ws, L.spl[p]), at<int32_t>(ws, L.gap[p]), at<NodeRec>(ws, L.nodes[p - 1]),
        at<NodeRec>(ws, L.nodes[p]), p, m);
    note_launch();
  }
  if (n_b > 0) {
    // split the sorted points by type; leaves get source ranges and query ranges,
    // node counts become source counts
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    int32_t* tile_cnt = at<int32_t>(ws, L.tile_cnt);
    k_src_tile_counts<<<(unsigned)tiles, kTypeThreads, 0, s>>>(pts, n, n_a, tile_cnt); note_launch();
    k_scan_tile_counts<<<1, 1024, 0, s>>>(tile_cnt, tiles); note_launch();
    k_split_types<<<(unsigned)tiles, kTypeThreads, 0, s>>>(pts, n, n_a, tile_cnt, at<float4>(ws, L.pts2),
                                                             at<int32_t>(ws, L.src_pos)); note_launch();
    k_leaf_types<<<grid_for(L.cap_nodes[0], 256, sms * 8), 256, 0, s>>>(
        at<NodeRec>(ws, L.nodes[0]), at<int32_t>(ws, L.src_pos), at<uint2>(ws, L.qrange), m); note_launch();
    for (int p = 1; p < L.n_planes; ++p)
      k_upper_counts<<<grid_for(L.cap_nodes[p] * 32, 256, sms * 16), 256, 0, s>>>(
          at<int32_t>(ws, L.spl[p]), at<NodeRec>(ws, L.nodes[p - 1]), at<NodeRec>(ws, L.nodes[p]), p, m);
    note_launch(L.n_planes - 1);
  }
  prof_end(kPhNodes, s);
}

}  // namespace

namespace {

__global__ void k_sort_prep(Meta* m) {
  for (int i = threadIdx.x; i < kMaxRadixPasses * kMaxRadixBins; i += blockDim.x) (&m->radix_hist[0][0])[i] = 0;
  if (threadIdx.x < kMaxRadixPasses) m->tile_ctr[threadIdx.x] = 0;
}

// Digit histograms of the first `passes` 8-bit digits of keys.
__global__ void __launch_bounds__(256) k_key_hist(const uint64_t* __restrict__ keys, int64_t n, int passes, Meta* m) {
  __shared__ uint32_t sh[kMaxRadixPasses][256];
  for (int i = threadIdx.x; i < kMaxRadixPasses * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(k >> (p * 8)) & 255], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
    const uint32_t v = (&sh[0][0])[i];
    if (v) atomicAdd(&m->radix_hist[i / 256][i % 256], v);
  }
}

}  // namespace

// Stable LSD sort of (k_a, index) by the low 8 * passes bits of k_a (passes even,
// at most 8): the sorted keys end in k_a and the indices in v_a; k_b and v_b are
// the ping-pong buffers; lookback holds passes * n_tiles * 256 words.  Uses the
// radix counters of the status block m (not during a build).
void launch_sort_u64(uint64_t* k_a, uint64_t* k_b, uint32_t* v_a, uint32_t* v_b, int64_t n, int passes,
                     uint32_t* lookback, cudaStream_t s, Meta* m) {
  const int sms = 152;
  const int64_t n_tiles = (n + kSortTile - 1) / kSortTile;
  k_sort_prep<<<1, 256, 0, s>>>(m); note_launch();
  k_key_hist<<<grid_for(n, 256, sms * 8), 256, 0, s>>>(k_a, n, passes, m); note_launch();
  k_radix_offsets<<<1, 32 * passes, 0, s>>>(m, passes, 256, 0); note_launch();
  const int64_t lb_words = n_tiles * 256 * passes;
  k_zero_u64<<<grid_for(lb_words / 2 + 1, 256, sms * 8), 256, 0, s>>>(
      reinterpret_cast<unsigned long long*>(lookback), (lb_words + 1) / 2); note_launch();
  const size_t smem = sizeof(SortSmem<8>);
  cudaFuncSetAttribute(k_onesweep<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const uint64_t* kin = k_a;
  const uint32_t* vin = nullptr;
  uint64_t* kout = k_b;
  uint32_t* vout = v_b;
  for (int p = 0; p < passes; ++p) {
    k_onesweep<8, false><<<(unsigned)n_tiles, kSortThreads, smem, s>>>(
        kin, vin, kout, vout, n, p, 8 * p, lookback + (size_t)p * n_tiles * 256, m, nullptr, nullptr, 0, nullptr, 0);
    note_launch();
    kin = kout;
    vin = vout;
    kout = (kout == k_b) ? k_a : k_b;
    vout = (vout == v_b) ? v_a : v_b;
  }
}

void launch_build(const float* d_xyz, int64_t n, float periodic_L, const Layout& L, char* ws, cudaStream_t s) {
  build_impl(d_xyz, n, nullptr, 0, periodic_L, L, ws, s);
}

void launch_build_sets(const float* d_src, int64_t n_src, const float* d_qry, int64_t n_qry, float periodic_L,
                       const Layout& L, char* ws, cudaStream_t s) {
  build_impl(d_src, n_src, d_qry, n_qry, periodic_L, L, ws, s);
}

}  // namespace jzt
