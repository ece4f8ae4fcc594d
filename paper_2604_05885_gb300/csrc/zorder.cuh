// The full-precision z-order of float32 points (Sec. II-A, Eq. msb and the
// comparator after it) and the node level on top of it (Sec. II-C, Eq. lvl).
//
// Every float32 value v is read as an unsigned 278-bit integer U(v): bit 277
// set for v >= 0 (zero counts as positive, -0 as +0) and the magnitude |v| 2^149
// (an exact integer for every normal and subnormal float32) below it, the
// magnitude's bits inverted for v < 0.  U is increasing in v, and the z-order of
// the comparator is the Morton order of the three U's, x most significant.
// zmsb() returns the position in U of the highest bit at which two values
// differ: 277 when the signs differ, -1 when the values are equal.  The
// comparator's msb(a, b) is zmsb(a, b) - 149 (EMAX = 128 for differing signs).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace jzt {

// Levels of the float order (Sec. II-C, Eq. lvl with d = 3): distinct points give
// (zmsb_k - 148) * 3 - k >= -446; equal points are made distinct by their sorted
// positions a < b: bit_length(a XOR b) + kZIndexLevel in [-478, -447]; the gaps
// before the first and after the last point carry kZSentinelLevel.
constexpr int kZIndexLevel = -479;
constexpr int kZSentinelLevel = 388;
constexpr int kZNoLevel = 32767;  // "no window" marker of the split kernels

__host__ __device__ __forceinline__ int zmsb(float a, float b) {
#ifdef __CUDA_ARCH__
  uint32_t ua = __float_as_uint(a), ub = __float_as_uint(b);
#else
  uint32_t ua, ub;
  memcpy(&ua, &a, 4);
  memcpy(&ub, &b, 4);
#endif
  if ((ua & 0x7fffffffu) == 0u) ua = 0u;  // -0 reads as +0
  if ((ub & 0x7fffffffu) == 0u) ub = 0u;
  if ((ua ^ ub) >> 31) return 277;        // signs differ
  const int ea = (int)((ua >> 23) & 0xffu), eb = (int)((ub >> 23) & 0xffu);
  // the magnitude of a normal value (exponent field e >= 1) is (2^23 + f) << (e - 1):
  // its leading bit sits at e + 22; a subnormal's (e = 0) is f itself
  if (ea != eb) return (ea > eb ? ea : eb) + 22;
  const uint32_t x = (ua ^ ub) & 0x7fffffu;
  if (x == 0u) return -1;
#ifdef __CUDA_ARCH__
  const int hb = 31 - __clz((int)x);
#else
  int hb = 31;
  while (!((x >> hb) & 1u)) --hb;
#endif
  return ea == 0 ? hb : hb + ea - 1;
}

// Dimension k compared by the comparator (largest zmsb, the lowest dimension on
// ties) and its zmsb; ms < 0 means the points are equal.
__host__ __device__ __forceinline__ int zdim(float ax, float ay, float az, float bx, float by, float bz, int* ms) {
  const int m0 = zmsb(ax, bx), m1 = zmsb(ay, by), m2 = zmsb(az, bz);
  int k = 0, mk = m0;
  if (m1 > mk) {
    k = 1;
    mk = m1;
  }
  if (m2 > mk) {
    k = 2;
    mk = m2;
  }
  *ms = mk;
  return k;
}

// Strict z-order of two points with their original indices as the last key
// (equal points keep index order, i.e. a stable sort of the input).
__device__ __forceinline__ bool zless(const float4& a, const float4& b) {
  int mk;
  const int k = zdim(a.x, a.y, a.z, b.x, b.y, b.z, &mk);
  if (mk < 0) return __float_as_uint(a.w) < __float_as_uint(b.w);
  const float va = k == 0 ? a.x : (k == 1 ? a.y : a.z);
  const float vb = k == 0 ? b.x : (k == 1 ? b.y : b.z);
  return va < vb;  // U is increasing in v, and the two differ in dimension k
}

// Level of two sorted points at positions ia < ib (Eq. lvl at full precision;
// equal points by their positions).
__device__ __forceinline__ int zlevel(const float4& a, const float4& b, int64_t ia, int64_t ib) {
  int mk;
  const int k = zdim(a.x, a.y, a.z, b.x, b.y, b.z, &mk);
  if (mk >= 0) return (mk - 148) * 3 - k;
  return 32 - __clz((int)((uint32_t)ia ^ (uint32_t)ib)) + kZIndexLevel;
}

}  // namespace jzt
