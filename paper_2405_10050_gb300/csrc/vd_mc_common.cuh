// vd_mc_common.cuh -- per-ray pieces of the Monte Carlo RayCast kernels
// (Section 3.1, Algorithm 3: rays from g = x_i with eta = {i}) that do not
// depend on where the candidates come from: the box faces as candidates, the
// per-ray candidate buffer and the binary64 recheck in canonical order.
#pragma once
#include "vd_ray_common.cuh"

namespace vd {

// Binary32 interval [tlo, thi] of the face t = (b - g_a) / u_a met along
// axis a (b = 1 if u_a > 0 else 0; face_bounds32); false if u_a == 0.
template <int D>
__device__ __forceinline__ bool mc_face(int a, const double (&u64)[D], const float (&u32)[D], const float (&g32)[D],
                                        int& s, float& tlo, float& thi) {
  double ua64 = 0.0;
  float ua = 0.f, va = 0.f;
#pragma unroll
  for (int q = 0; q < D; ++q)
    if (q == a) {
      ua64 = u64[q];
      ua = u32[q];
      va = g32[q];
    }
  s = face_bounds32(ua, ua64, va, tlo, thi);
  return s >= 0;
}

// Box faces of a ray from g as candidates: returns an upper bound T of the
// smallest face t and appends to (cb, ct) the faces whose lower bound is
// <= T.  Sets `overflow` if they do not fit.
template <int D>
__device__ __forceinline__ float mc_faces(const double (&u64)[D], const float (&u32)[D], const float (&g32)[D], int d,
                                          int32_t* cb, float* ct, int& nc, int cap, bool& overflow) {
  float T = INFINITY;
  int s;
  float tlo, thi;
  for (int a = 0; a < d; ++a)
    if (mc_face<D>(a, u64, u32, g32, s, tlo, thi)) T = fminf(T, thi);
  for (int a = 0; a < d; ++a)
    if (mc_face<D>(a, u64, u32, g32, s, tlo, thi) && tlo <= T) {
      if (nc < cap) {
        cb[nc] = face_id(a, s);
        ct[nc] = tlo;
        ++nc;
      } else {
        overflow = true;
      }
    }
  return T;
}

// Keeps candidate id with lower bound tlo if it can still beat T; entries
// the bound has since excluded are dropped first.  Returns false when the
// buffer is full of live entries (the ray must be finished elsewhere).
__device__ __forceinline__ bool mc_push(int32_t id, float tlo, float T, int32_t* cb, float* ct, int& nc, int cap) {
  if (!(tlo <= T)) return true;
  if (nc == cap) {
    int m = 0;
    for (int q = 0; q < cap; ++q)
      if (ct[q] <= T) {
        cb[m] = cb[q];
        ct[m] = ct[q];
        ++m;
      }
    nc = m;
  }
  if (nc == cap) return false;
  cb[nc] = id;
  ct[nc] = tlo;
  ++nc;
  return true;
}

// Binary64 recheck of the buffered candidates whose lower bound is <= T:
// t_j = |w|^2 / (2 u.w) with w = x_j - g (v = g), canonical operation order,
// den > 0 strictly; faces t = (b - g_a) / u_a.  Writes the argmin under the
// order (t, class, id) as a generator id and its t.
template <int D>
__device__ __forceinline__ void mc_recheck(const double* X, int d, const double (&g64)[D], const double (&u64)[D],
                                           const int32_t* cb, const float* ct, int nc, float T, int32_t& hit,
                                           double& tbest, unsigned long long& n_rech) {
  double bt = INFINITY;
  int bc = 2, bk = 0;
  for (int q = 0; q < nc; ++q) {
    if (!(ct[q] <= T)) continue;
    const int32_t id = cb[q];
    ++n_rech;
    if (id >= 0) {
      double w[D], dn = 0.0, ww = 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a) w[a] = a < d ? __dadd_rn(X[(int64_t)id * d + a], -g64[a]) : 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a < d) dn = __dadd_rn(dn, __dmul_rn(u64[a], w[a]));
      if (!(dn > 0.0)) continue;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a < d) ww = __dadd_rn(ww, __dmul_rn(w[a], w[a]));
      const double t = __ddiv_rn(ww, __dmul_rn(2.0, dn));
      if (better(t, 0, id, bt, bc, bk)) {
        bt = t;
        bc = 0;
        bk = id;
      }
    } else {
      const int a = face_axis(id), s = face_side(id);
      double ua = 0.0, va = 0.0;
#pragma unroll
      for (int q2 = 0; q2 < D; ++q2)
        if (q2 == a) {
          ua = u64[q2];
          va = g64[q2];
        }
      const double t = __ddiv_rn(__dadd_rn(s ? 1.0 : 0.0, -va), ua);
      if (better(t, 1, 2 * a + s, bt, bc, bk)) {
        bt = t;
        bc = 1;
        bk = 2 * a + s;
      }
    }
  }
  hit = gen_from_key(bc, bk);
  tbest = bt;
}

// Error constants of the tensor-core screening: |den_mma - u.w| <= a1 |w| + a0
// for |u| = 1, where the MMA multiplies the fp16 roundings of binary32 u and
// w and accumulates in fp32:
//   fp16 (and before it binary32) rounding of each u_k and w_k: relative
//   2^-11 + 2^-24, plus an absolute 2^-25 below the fp16 normal range, which
//   over the d terms adds at most sqrt(d) 2^-25 (|w| + 1);
//   products of two fp16 values are exact in fp32; the sum of the 16 products
//   is charged 2^-16 of sum |u_k w_k| <= |w|, far above the 16 x 2^-23 of any
//   fp32 accumulation order or rounding mode.
struct TcBound {
  float a1, a0;
};
__device__ __forceinline__ TcBound tc_bound(int D) {
  const float sq = sqrtf((float)D);
  return {1.1f * (0x1p-10f + 0x1p-22f + 0x1p-16f + sq * 0x1p-25f), 1.1f * sq * 0x1p-25f};
}

}  // namespace vd
