// vd_dev.cuh -- device helpers of libvd: generator ids, the counter-based
// direction draw, canonical binary64 arithmetic and warp utilities.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "vd_internal.h"

namespace vd {

__host__ __device__ inline int32_t face_id(int a, int s) { return -(2 * a + s + 1); }
__host__ __device__ inline int face_axis(int32_t id) { return (-id - 1) >> 1; }
__host__ __device__ inline int face_side(int32_t id) { return (-id - 1) & 1; }

constexpr unsigned kFull = 0xffffffffu;
constexpr float kU32 = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of binary32

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the
// two 32x32->64 multiplications with key bumps by the Weyl constants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// binary32 log of x in (0,1]: x = m 2^e, m in [sqrt(1/2), sqrt(2)),
// ln m = 2 artanh(s), s = (m-1)/(m+1), series through s^11; e ln2 with ln2
// split into a 16-bit high part and a low part.  Every operation rounds
// separately (no contraction), so the result is bit-reproducible.
__device__ __forceinline__ float ln32(float x) {
  const uint32_t b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fadd_rn(m, -1.0f), __fadd_rn(m, 1.0f));
  const float z = __fmul_rn(s, s);
  float p = 0x1.745d18p-4f;
  p = __fadd_rn(__fmul_rn(p, z), 0x1.c71c72p-4f);
  p = __fadd_rn(__fmul_rn(p, z), 0x1.24924ap-3f);
  p = __fadd_rn(__fmul_rn(p, z), 0x1.99999ap-3f);
  p = __fadd_rn(__fmul_rn(p, z), 0x1.555556p-2f);
  p = __fadd_rn(__fmul_rn(p, z), 1.0f);
  const float lnm = __fmul_rn(__fadd_rn(s, s), p);
  const float fe = __int2float_rn(e);
  const float lo = __fmul_rn(fe, 0x1.7f7d1cp-20f);
  const float hi = __fmul_rn(fe, 0x1.62e4p-1f);
  return __fadd_rn(hi, __fadd_rn(lo, lnm));
}

// cos and sin of 2 pi a / 2^24 (a < 2^24): exact octant reduction on the
// integer angle, Taylor series on [0, pi/4].
__device__ __forceinline__ void sincos2pi24(uint32_t a, float& c, float& s) {
  const uint32_t q = a >> 21, f = a & 0x1fffffu;
  const uint32_t g = (q & 1u) ? (0x200000u - f) : f;
  const float phi = __fmul_rn(0x1.921fb6p+2f, __fmul_rn(__uint2float_rn(g), 0x1p-24f));
  const float z = __fmul_rn(phi, phi);
  float ps = 0x1.71de3ap-19f;
  ps = __fadd_rn(__fmul_rn(ps, z), -0x1.a01a02p-13f);
  ps = __fadd_rn(__fmul_rn(ps, z), 0x1.111112p-7f);
  ps = __fadd_rn(__fmul_rn(ps, z), -0x1.555556p-3f);
  ps = __fadd_rn(__fmul_rn(ps, z), 1.0f);
  const float S = __fmul_rn(phi, ps);
  float pc = -0x1.27e4fcp-22f;
  pc = __fadd_rn(__fmul_rn(pc, z), 0x1.a01a02p-16f);
  pc = __fadd_rn(__fmul_rn(pc, z), -0x1.6c16c2p-10f);
  pc = __fadd_rn(__fmul_rn(pc, z), 0x1.555556p-5f);
  pc = __fadd_rn(__fmul_rn(pc, z), -0.5f);
  pc = __fadd_rn(__fmul_rn(pc, z), 1.0f);
  const float C = pc;
  switch (q) {
    case 0: c = C; s = S; break;
    case 1: c = S; s = C; break;
    case 2: c = -S; s = C; break;
    case 3: c = -C; s = S; break;
    case 4: c = -C; s = -S; break;
    case 5: c = -S; s = -C; break;
    case 6: c = S; s = -C; break;
    default: c = C; s = -S; break;
  }
}

__device__ __forceinline__ void box_muller32(uint32_t x0, uint32_t x1, float& z0, float& z1) {
  const float U = __fmul_rn(__uint2float_rn((x0 >> 9) * 2u + 1u), 0x1p-24f);
  const float r = __fsqrt_rn(__fmul_rn(-2.0f, ln32(U)));
  float c, s;
  sincos2pi24(x1 >> 8, c, s);
  z0 = __fmul_rn(r, c);
  z1 = __fmul_rn(r, s);
}

// Direction of ray k of cell i of point set `set` (Section 3.1: normalised
// Gaussian).  Philox counter (block, k, i, set), key (seed lo, seed hi);
// binary32 Box-Muller, binary64 u = z * (1 / sqrt(sum z^2)).
template <int D>
__device__ __forceinline__ void mc_direction(uint64_t seed, uint32_t set, uint32_t cell, uint32_t ray, int d,
                                             double u[D]) {
  float z[(D + 3) / 4 * 4];
#pragma unroll
  for (int blk = 0; blk < (D + 3) / 4; ++blk) {
    uint32_t c[4] = {(uint32_t)blk, ray, cell, set};
    philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    box_muller32(c[0], c[1], z[4 * blk + 0], z[4 * blk + 1]);
    box_muller32(c[2], c[3], z[4 * blk + 2], z[4 * blk + 3]);
  }
  // sum of the squares from the left (d >= 1); the first term is taken as
  // it is, since 0 + z_0^2 = z_0^2 exactly (z_0^2 >= +0)
  const double z0 = (double)z[0];
  double ss = __dmul_rn(z0, z0);
#pragma unroll
  for (int k = 1; k < D; ++k)
    if (k < d) {
      const double zk = (double)z[k];
      ss = __dadd_rn(ss, __dmul_rn(zk, zk));
    }
  const double inv = __drcp_rn(__dsqrt_rn(ss));
#pragma unroll
  for (int k = 0; k < D; ++k) u[k] = (k < d) ? __dmul_rn((double)z[k], inv) : 0.0;
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Total order used everywhere: (t, class, key) with class 0 = node (key =
// id), class 1 = face (key = 2a+s).
__device__ __forceinline__ bool better(double t, int cls, int key, double bt, int bcls, int bkey) {
  if (t < bt) return true;
  if (t > bt) return false;
  if (cls != bcls) return cls < bcls;
  return key < bkey;
}

__device__ __forceinline__ void warp_argmin(double& t, int& cls, int& key) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const double t2 = __shfl_xor_sync(kFull, t, o);
    const int c2 = __shfl_xor_sync(kFull, cls, o);
    const int k2 = __shfl_xor_sync(kFull, key, o);
    if (better(t2, c2, k2, t, cls, key)) {
      t = t2;
      cls = c2;
      key = k2;
    }
  }
}

__device__ __forceinline__ int32_t gen_from_key(int cls, int key) {
  return cls == 0 ? key : (cls == 1 ? -(key + 1) : kNoId);
}

// Bitonic sort of (key, val) across the 32 lanes, ascending in key.
__device__ __forceinline__ void warp_sort(float& k, int& v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const float k2 = __shfl_xor_sync(kFull, k, stride);
      const int v2 = __shfl_xor_sync(kFull, v, stride);
      const bool up = ((lane & size) == 0);
      const bool lower = ((lane & stride) == 0);
      const bool take = lower ? (up ? (k2 < k || (k2 == k && v2 < v)) : (k2 > k || (k2 == k && v2 > v)))
                              : (up ? (k2 > k || (k2 == k && v2 > v)) : (k2 < k || (k2 == k && v2 < v)));
      if (take) {
        k = k2;
        v = v2;
      }
    }
  }
}

__device__ __forceinline__ float f32_down(double x) { return __double2float_rd(x); }
__device__ __forceinline__ float f32_up(double x) { return __double2float_ru(x); }

}  // namespace vd
