// vd_ray_common.cuh -- binary32 screening helpers shared by the RayCast
// kernels: the conservative ball of the current bound, the candidate-list
// distance and its lower bound, and the box-clipped reach of the ball.
#pragma once
#include "vd_dev.cuh"
#include "vd_internal.h"

namespace vd {

// Binary32 bounds [tlo, thi] of t = (b - v_a) / u_a, where the ray meets the
// box face of axis a on the side it moves to (b = 1 if u_a > 0, else 0), from
// ua = u_a rounded to binary32 and va = v_a rounded to binary32.  Returns the
// side (1: b = 1, 0: b = 0), or -1 if u_a = 0 (the ray never meets the face).
// ua has u_a's sign; it is 0 for 0 < |u_a| <= 2^-150 too, and there binary32
// bounds nothing (the face may still be near if v_a is within ~|u_a| of b):
// the face then gets (-inf, inf) and so is always rechecked in binary64.
__device__ __forceinline__ int face_bounds32(float ua, double ua64, float va, float& tlo, float& thi) {
  if (ua == 0.f) {
    if (ua64 == 0.0) return -1;
    tlo = -INFINITY;
    thi = INFINITY;
    return ua64 > 0.0 ? 1 : 0;
  }
  const int s = ua > 0.f ? 1 : 0;
  const float nf = (s ? 1.f : 0.f) - va;
  const float nfs = s ? nf : -nf;  // t = nfs / |u_a|
  const float ef = 1.01f * kU32 * (fabsf(va) + fabsf(nf)) + 1e-38f;
  const float au = fabsf(ua);
  const float lo_n = nfs - ef, hi_n = nfs + ef;
  tlo = lo_n >= 0.f ? lo_n / (au * (1.f + 2.f * kU32)) * (1.f - 4.f * kU32)
                    : lo_n / (au * (1.f - 2.f * kU32)) * (1.f + 4.f * kU32);
  thi = hi_n >= 0.f ? hi_n / (au * (1.f - 2.f * kU32)) * (1.f + 4.f * kU32)
                    : hi_n / (au * (1.f + 2.f * kU32)) * (1.f - 4.f * kU32);
  return s;
}

// Conservative binary32 ball: every point within distance rho of the exact
// centre c = v + T u satisfies |y - c32|^2 <= lim2.
template <int D>
struct Ball {
  float c[D];
  float lim2;
  float rho_hi;  // upper bound of the exact radius |g - c|
};

template <int D>
__device__ __forceinline__ void make_ball(const float g[D], const float p[D], const float u[D], float T, float B,
                                          Ball<D>& b) {
  // c = g + p + T u, rho = |p + T u|; absolute error of each coordinate is
  // below 4 u_32 (|g| + |p| + T) and of rho below 4 sqrt(D) u_32 (...).
  float r2 = 0.f, pm = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float q = fmaf(T, u[k], p[k]);
    b.c[k] = g[k] + q;
    r2 = fmaf(q, q, r2);
    pm = fmaxf(pm, fabsf(p[k]));
  }
  const float eps = 8.f * (float)D * kU32 * (B + pm + T) + 1e-30f;
  const float rho = sqrtf(r2) * (1.f + 4.f * (float)D * kU32) + eps;
  b.lim2 = rho * rho * (1.f + 4.f * (float)D * kU32) + 1e-37f;
  b.rho_hi = rho;
  if (!(T < INFINITY)) {
    b.lim2 = INFINITY;
    b.rho_hi = INFINITY;
  }
}

// Candidate lists: ww32 = sum_k fma-chain (x32_k - g32_k)^2 over k = 0..D-1;
// the same function orders the lists and is evaluated during the scan.
template <int D>
__device__ __forceinline__ float ww32_of(const float* xs, int stride, const float* g32, int d) {
  float ww = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float w = (k < d) ? xs[k * stride] - g32[k] : 0.f;
    ww = fmaf(w, w, ww);
  }
  return ww;
}

// Lower bound of the exact |x - g|^2 from ww32 (w32 components within EW of
// the exact ones, gamma_D for the FMA chain).
__device__ __forceinline__ float true_d2_lower(float ww, float gam, float EW, int D) {
  const float l = ww * (1.f - 2.f * gam) - 2.02f * sqrtf((float)D) * EW * sqrtf(ww) - (float)D * EW * EW;
  return fmaxf(l, 0.f);
}

// A binary32 squared distance ww32 >= ww_exit(f) implies
// true_d2_lower(ww32) >= f: with a = 1 - 2 gam, b = 2.02 sqrt(D) EW,
// c = D EW^2 the bound is a s^2 - b s - c at s = sqrt(ww32), increasing for
// s > b / (2a); its root for f, squared, is inflated by 2^-12 to cover the
// rounding of this evaluation.
__device__ __forceinline__ float ww_exit(float f, float gam, float EW, int D) {
  if (!(f < INFINITY)) return INFINITY;
  const float a = 1.f - 2.f * gam, b = 2.02f * sqrtf((float)D) * EW, c = (float)D * EW * EW;
  const float s = (b + sqrtf(fmaf(b, b, 4.f * a * (c + fmaxf(f, 0.f))))) / (2.f * a);
  return s * s * (1.f + 0x1p-12f);
}

// Squared radius around g that holds every node of the ball: nodes lie in
// the node box, so only the part of the ball inside it matters; the farthest
// point from g of that part is bounded through its axis-aligned box
// [max(c - rho, lo), min(c + rho, hi)], and by the ball's diameter 2 rho
// (the ball passes through g).  Returns 0 when the ball misses the box.
template <int D>
__device__ __forceinline__ float far_radius2(const TreeView& tr, const Ball<D>& b, const float* g32) {
  if (!(b.rho_hi < INFINITY)) return INFINITY;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (k < tr.d) {
      const float L = fmaxf(b.c[k] - b.rho_hi, tr.root_lo[k]);
      const float H = fminf(b.c[k] + b.rho_hi, tr.root_hi[k]);
      if (L > H) return 0.f;
      const float m = fmaxf(fabsf(L - g32[k]), fabsf(H - g32[k])) * (1.f + 4.f * kU32) + 2.f * kU32 * tr.coord_abs;
      s = fmaf(m, m, s);
    }
  }
  s *= 1.f + 4.f * (float)D * kU32;
  return fminf(s, 4.f * b.rho_hi * b.rho_hi * (1.f + 4.f * kU32));
}


// ---- ray and node loads shared by the RayCast kernels ----

// Origin v and direction u of ray r of the source.
template <int D>
__device__ __forceinline__ void load_vu(const TreeView& tr, const RaySource& rs, int64_t r, double v[D], double u[D]) {
  const int d = tr.d;
  if (rs.mode == 0) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      v[k] = k < d ? rs.origins[r * d + k] : 0.0;
      u[k] = k < d ? rs.dirs[r * d + k] : 0.0;
    }
  } else {
    const int32_t cell = rs.mc_cell ? rs.mc_cell[r] : (int32_t)(r / rs.mc_rpc);
    const int32_t k = rs.mc_cell ? rs.mc_ray[r] : (int32_t)(r % rs.mc_rpc);
    mc_direction<D>(rs.seed, rs.set, (uint32_t)cell, (uint32_t)k, d, u);
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = k < d ? tr.X[(int64_t)cell * d + k] : 0.0;
  }
}

// Loads ray r of the source: origin v, direction u, eta (m ids, eta[0] = g).
template <int D>
__device__ __forceinline__ void load_ray(const TreeView& tr, const RaySource& rs, int64_t r, double v[D], double u[D],
                                         int32_t eta[D + 1], int& m) {
  load_vu<D>(tr, rs, r, v, u);
  if (rs.mode == 0) {
    m = 0;
    for (int q = 0; q < rs.eta_stride && q < D + 1; ++q) {
      const int32_t e = rs.eta[r * rs.eta_stride + q];
      if (e == kNoId) break;
      eta[m++] = e;
    }
  } else {
    eta[0] = rs.mc_cell ? rs.mc_cell[r] : (int32_t)(r / rs.mc_rpc);
    m = 1;
  }
}

__device__ __forceinline__ int64_t out_pos(const RaySource& rs, const RayOut& ro, int64_t r) {
  if (rs.mode == 0 || rs.mc_cell == nullptr) return r;
  return (int64_t)rs.mc_cell[r] * ro.mc_rpc + rs.mc_ray[r];
}

// Binary32 coordinates of node id (zeros when !valid): from the rows padded
// to 16-byte vectors where they exist (d <= 8), else one by one.
template <int D>
__device__ __forceinline__ void load_x32(const TreeView& tr, int32_t id, bool valid, float (&x)[D]) {
  if constexpr (D <= 8) {
    if (tr.X32v != nullptr) {
      constexpr int Q = (D + 3) / 4;
      const float4* row = tr.X32v + (int64_t)id * tr.x32q;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const float4 f = (valid && j < tr.x32q) ? row[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float e[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (4 * j + k < D) x[4 * j + k] = e[k];
      }
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = (valid && k < tr.d) ? tr.X32[(int64_t)id * tr.d + k] : 0.f;
}

// Upper bound of the norm from the binary32 sum of squares ww, with the same
// margin (1 + gam) as sqrtf(ww) (1 + gam) plus 2^-20 for the reciprocal square
// root (documented error 2 ulp) and the product; 0 for ww = 0, inf for
// ww = inf.
__device__ __forceinline__ float norm_up(float ww, float gam) {
  const float s = ww < INFINITY ? fmaxf(ww * rsqrtf(ww), 0.f) : INFINITY;
  return s * (1.f + gam + 0x1p-20f);
}

}  // namespace vd
