// FoF catalogue reduction (Sec. IV-B): after the group labels, the points are
// brought into group order -- a stable sort of the z-ordered points by the z
// position of their group's root (the member with the lowest z position), so
// roots keep their z order and every group is a contiguous block in z order --
// and per group of at least min_count points the mass, the centre of mass, the
// inertia radius and the centre-of-mass velocity are reduced.
//
// Scratch lives in the interaction-list arena, which the FoF walk no longer
// needs once the labels are written.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "common.cuh"

namespace jzt {

int fail_msg(int code, const std::string& msg);  // api.cu

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCatThreads = 256;
constexpr int kCatPer = kScanTile / kCatThreads;

int cat_grid(int64_t work, int threads, int max_blocks) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

__device__ __forceinline__ uint32_t cat_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t s_w[kCatThreads / 32];
  __shared__ uint32_t s_tot;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane_id() >= o) inc += y;
  }
  if (lane_id() == 31) s_w[warp_id()] = inc;
  __syncthreads();
  if (warp_id() == 0) {
    uint32_t w = lane_id() < kCatThreads / 32 ? s_w[lane_id()] : 0u, wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, wi, o);
      if (lane_id() >= o) wi += y;
    }
    if (lane_id() < kCatThreads / 32) s_w[lane_id()] = wi - w;
    if (lane_id() == 31) s_tot = wi;
  }
  __syncthreads();
  const uint32_t res = s_w[warp_id()] + inc - v;
  *total = s_tot;
  __syncthreads();
  return res;
}

// sort key of z position i: its root's z position
__global__ void k_cat_keys(const int32_t* __restrict__ ig_pt, int64_t n, uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = (uint64_t)(uint32_t)ig_pt[i];
}

// group starts in group order: position 0 and every change of root
__device__ __forceinline__ bool is_start(const uint64_t* keys, int64_t i) { return i == 0 || keys[i] != keys[i - 1]; }

__global__ void __launch_bounds__(kCatThreads) k_cat_start_counts(const uint64_t* __restrict__ keys, int64_t n,
                                                                  int32_t* tile_cnt) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kCatPer;
  uint32_t c = 0;
#pragma unroll
  for (int e = 0; e < kCatPer; ++e) c += (base + e < n && is_start(keys, base + e)) ? 1u : 0u;
  uint32_t total;
  (void)cat_excl_scan(c, &total);
  if (threadIdx.x == 0) tile_cnt[blockIdx.x] = (int32_t)total;
}

// gstart[g] = first position of group g in group order; gstart[G] = n, *n_groups = G
__global__ void __launch_bounds__(kCatThreads) k_cat_starts(const uint64_t* __restrict__ keys, int64_t n,
                                                            const int32_t* __restrict__ tile_off, int64_t n_tiles,
                                                            int32_t* __restrict__ gstart, int64_t* n_groups) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kCatPer;
  uint32_t c = 0;
#pragma unroll
  for (int e = 0; e < kCatPer; ++e) c += (base + e < n && is_start(keys, base + e)) ? 1u : 0u;
  uint32_t total;
  int32_t r = tile_off[blockIdx.x] + (int32_t)cat_excl_scan(c, &total);
#pragma unroll
  for (int e = 0; e < kCatPer; ++e) {
    const int64_t i = base + e;
    if (i < n && is_start(keys, i)) gstart[r++] = (int32_t)i;
  }
  if (blockIdx.x == n_tiles - 1 && threadIdx.x == 0) {
    const int64_t G = (int64_t)tile_off[blockIdx.x] + (int64_t)total;
    gstart[G] = (int32_t)n;
    *n_groups = G;
  }
}

// kept groups (count >= min_count): per tile of groups, then their output slots
__global__ void __launch_bounds__(kCatThreads) k_cat_kept_counts(const int32_t* __restrict__ gstart,
                                                                 const int64_t* __restrict__ n_groups, int min_count,
                                                                 int32_t* tile_cnt) {
  const int64_t G = *n_groups;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kCatPer;
  uint32_t c = 0;
#pragma unroll
  for (int e = 0; e < kCatPer; ++e) {
    const int64_t g = base + e;
    c += (g < G && gstart[g + 1] - gstart[g] >= min_count) ? 1u : 0u;
  }
  uint32_t total;
  (void)cat_excl_scan(c, &total);
  if (threadIdx.x == 0) tile_cnt[blockIdx.x] = (int32_t)total;
}

__global__ void __launch_bounds__(kCatThreads) k_cat_kept_index(const int32_t* __restrict__ gstart,
                                                                const int64_t* __restrict__ n_groups, int min_count,
                                                                const int32_t* __restrict__ tile_off, int64_t n_tiles,
                                                                int32_t* __restrict__ out_idx, int64_t* n_kept,
                                                                int64_t cap, Meta* m) {
  const int64_t G = *n_groups;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kCatPer;
  uint32_t c = 0;
#pragma unroll
  for (int e = 0; e < kCatPer; ++e) {
    const int64_t g = base + e;
    c += (g < G && gstart[g + 1] - gstart[g] >= min_count) ? 1u : 0u;
  }
  uint32_t total;
  int32_t r = tile_off[blockIdx.x] + (int32_t)cat_excl_scan(c, &total);
#pragma unroll
  for (int e = 0; e < kCatPer; ++e) {
    const int64_t g = base + e;
    if (g < G) out_idx[g] = (gstart[g + 1] - gstart[g] >= min_count) ? r++ : -1;
  }
  if (blockIdx.x == n_tiles - 1 && threadIdx.x == 0) {
    const int64_t K = (int64_t)tile_off[blockIdx.x] + (int64_t)total;
    *n_kept = K;
    if (K > cap) set_error(m, JZT_ERR_CAPACITY, kStageLeaf);
  }
}

// exclusive scan of tile counts in place (one block)
__global__ void __launch_bounds__(kCatThreads) k_cat_scan_tiles(int32_t* tile_cnt, int64_t n_tiles) {
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < n_tiles; b += kCatThreads) {
    const int64_t i = b + threadIdx.x;
    const uint32_t v = i < n_tiles ? (uint32_t)tile_cnt[i] : 0u;
    uint32_t total;
    const uint32_t ex = cat_excl_scan(v, &total);
    if (i < n_tiles) tile_cnt[i] = carry + (int32_t)ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += (int32_t)total;
    __syncthreads();
  }
}

// original index of each point in group order
__global__ void k_cat_order(const float4* __restrict__ pts, const uint32_t* __restrict__ zpos, int64_t n,
                            int32_t* __restrict__ order) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    order[i] = __float_as_int(pts[zpos[i]].w);
}

__device__ __forceinline__ double wrap_d(double d, double L) { return d - L * rint(d / L); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// One warp per group (grid-stride): float64 sums in a fixed order, so the result
// does not depend on scheduling.  Positions are taken relative to the root (the
// group's first point in group order) by the minimum image when periodic.
template <bool PER>
__global__ void __launch_bounds__(256) k_cat_stats(const float4* __restrict__ pts, const uint32_t* __restrict__ zpos,
                                                   const int32_t* __restrict__ gstart, const int64_t* __restrict__ n_groups,
                                                   const int32_t* __restrict__ out_idx, const int32_t* __restrict__ minorig,
                                                   const float* __restrict__ vel, float pmass, float L, int64_t cap,
                                                   jzt_group* __restrict__ out) {
  const int64_t G = *n_groups;
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
    const int32_t o = out_idx[g];
    if (o < 0 || o >= cap) continue;
    const int64_t s = gstart[g], e = gstart[g + 1];
    const float4 r = pts[zpos[s]];
    const double rx = r.x, ry = r.y, rz = r.z, Ld = L;
    double sx = 0, sy = 0, sz = 0, vx = 0, vy = 0, vz = 0;
    for (int64_t j = s + lane; j < e; j += 32) {
      const float4 p = pts[zpos[j]];
      double dx = (double)p.x - rx, dy = (double)p.y - ry, dz = (double)p.z - rz;
      if (PER) {
        dx = wrap_d(dx, Ld);
        dy = wrap_d(dy, Ld);
        dz = wrap_d(dz, Ld);
      }
      sx += dx;
      sy += dy;
      sz += dz;
      if (vel) {
        const int64_t oi = __float_as_int(p.w);
        vx += vel[3 * oi];
        vy += vel[3 * oi + 1];
        vz += vel[3 * oi + 2];
      }
    }
    const double cnt = (double)(e - s);
    const double mx = warp_sum(sx) / cnt, my = warp_sum(sy) / cnt, mz = warp_sum(sz) / cnt;
    vx = warp_sum(vx);
    vy = warp_sum(vy);
    vz = warp_sum(vz);
    double q = 0;
    for (int64_t j = s + lane; j < e; j += 32) {
      const float4 p = pts[zpos[j]];
      double dx = (double)p.x - rx, dy = (double)p.y - ry, dz = (double)p.z - rz;
      if (PER) {
        dx = wrap_d(dx, Ld);
        dy = wrap_d(dy, Ld);
        dz = wrap_d(dz, Ld);
      }
      dx -= mx;
      dy -= my;
      dz -= mz;
      q += dx * dx + dy * dy + dz * dz;
    }
    q = warp_sum(q);
    if (lane == 0) {
      double cx = rx + mx, cy = ry + my, cz = rz + mz;
      if (PER) {
        cx -= Ld * floor(cx / Ld);
        cy -= Ld * floor(cy / Ld);
        cz -= Ld * floor(cz / Ld);
      }
      jzt_group gr;
      gr.label = minorig[zpos[s]];
      gr.count = (int32_t)(e - s);
      gr.offset = s;
      gr.mass = (float)(cnt * (double)pmass);
      gr.x_cm[0] = (float)cx;
      gr.x_cm[1] = (float)cy;
      gr.x_cm[2] = (float)cz;
      gr.v_cm[0] = (float)(vx / cnt);
      gr.v_cm[1] = (float)(vy / cnt);
      gr.v_cm[2] = (float)(vz / cnt);
      gr.r_inertia = (float)sqrt(q / cnt);
      out[o] = gr;
    }
  }
}

}  // namespace

// Scratch bytes in the arena for n points.
size_t catalogue_scratch_bytes(int64_t n) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  return 8 * (size_t)n * 2 + 4 * (size_t)n * 2 + 4 * (size_t)(n + 1) + 4 * (size_t)n + 4 * (size_t)(tiles + 1) +
         4 * (size_t)(tiles + 1) + 64 + 6 * 256;
}

int launch_catalogue(const Layout& L, char* ws, float periodic_L, const float* d_vel, int min_count,
                     float particle_mass, int32_t* d_order, jzt_group* d_groups, int64_t cap_groups,
                     int64_t* d_n_groups, cudaStream_t s) {
  const int64_t n = L.n;
  Meta* m = at<Meta>(ws, L.meta);
  const int sms = 152;
  // scratch in the arena (free after the FoF walk)
  char* a = at<char>(ws, L.arena);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = a + off;
    off = (off + bytes + 255) & ~(size_t)255;
    return p;
  };
  uint64_t* k_a = reinterpret_cast<uint64_t*>(take(8 * (size_t)n));
  uint64_t* k_b = reinterpret_cast<uint64_t*>(take(8 * (size_t)n));
  uint32_t* v_a = reinterpret_cast<uint32_t*>(take(4 * (size_t)n));
  uint32_t* v_b = reinterpret_cast<uint32_t*>(take(4 * (size_t)n));
  int32_t* gstart = reinterpret_cast<int32_t*>(take(4 * (size_t)(n + 1)));
  int32_t* out_idx = reinterpret_cast<int32_t*>(take(4 * (size_t)n));
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  int32_t* tile_a = reinterpret_cast<int32_t*>(take(4 * (size_t)(tiles + 1)));
  int32_t* tile_b = reinterpret_cast<int32_t*>(take(4 * (size_t)(tiles + 1)));
  int64_t* n_groups = reinterpret_cast<int64_t*>(take(64));
  if (off > sizeof(IEntry) * (size_t)L.cap_ilist)
    return fail_msg(JZT_ERR_WORKSPACE, "workspace too small for the catalogue scratch (" + std::to_string(off) +
                                           " bytes of interaction-list space needed)");
  const int32_t* ig_pt = at<int32_t>(ws, L.ig_pt);
  const float4* pts = at<float4>(ws, L.pts);
  // group order: stable sort of z positions by root z position (roots < 2^31: 4 passes of 8 bits)
  k_cat_keys<<<cat_grid(n, 256, sms * 8), 256, 0, s>>>(ig_pt, n, k_a); note_launch();
  launch_sort_u64(k_a, k_b, v_a, v_b, n, 4, at<uint32_t>(ws, L.lookback), s, m);
  k_cat_order<<<cat_grid(n, 256, sms * 8), 256, 0, s>>>(pts, v_a, n, d_order); note_launch();
  // groups
  k_cat_start_counts<<<(unsigned)tiles, kCatThreads, 0, s>>>(k_a, n, tile_a); note_launch();
  k_cat_scan_tiles<<<1, kCatThreads, 0, s>>>(tile_a, tiles); note_launch();
  k_cat_starts<<<(unsigned)tiles, kCatThreads, 0, s>>>(k_a, n, tile_a, tiles, gstart, n_groups);
  note_launch();
  // kept groups (the number of groups is at most n: size the grid for n)
  k_cat_kept_counts<<<(unsigned)tiles, kCatThreads, 0, s>>>(gstart, n_groups, min_count, tile_b); note_launch();
  k_cat_scan_tiles<<<1, kCatThreads, 0, s>>>(tile_b, tiles); note_launch();
  k_cat_kept_index<<<(unsigned)tiles, kCatThreads, 0, s>>>(gstart, n_groups, min_count, tile_b, tiles, out_idx,
                                                           d_n_groups, cap_groups, m);
  note_launch();
  if (periodic_L > 0.0f)
    k_cat_stats<true><<<sms * 16, 256, 0, s>>>(pts, v_a, gstart, n_groups, out_idx, at<int32_t>(ws, L.minorig), d_vel,
                                              particle_mass, periodic_L, cap_groups, d_groups);
  else
    k_cat_stats<false><<<sms * 16, 256, 0, s>>>(pts, v_a, gstart, n_groups, out_idx, at<int32_t>(ws, L.minorig),
                                               d_vel, particle_mass, 0.0f, cap_groups, d_groups);
  note_launch();
  return JZT_OK;
}

}  // namespace jzt
