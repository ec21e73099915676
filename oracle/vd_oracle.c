/*
 * vd_oracle.c -- plain, slow, FP64 CPU oracle for the exact Voronoi RayCast,
 * the exhaustive vertex traversal and the Monte Carlo cell integrals of
 * Sikorski & Heida, "Voronoi Graph" (arXiv 2405.10050).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant table with the
 * CUDA library.
 *
 * Everything is brute force: every ray is tested against every node.  All
 * floating point follows IEEE binary64 (binary32 for the Gaussian draw),
 * round to nearest, no contraction (build with -ffp-contract=off), in the
 * operation order written below.  That order is the canonical definition the
 * GPU path reproduces.
 *
 * Generator ids: nodes are 0..N-1; the faces of the unit box [0,1]^d are
 * pseudo-generators with negative ids, -(2a+s+1) for axis a and side s
 * (s=0: x_a=0, s=1: x_a=1).  "No generator" is INT32_MIN.
 *
 * Pins: every routine is checked in tests/test_oracle_*.py against things
 * other than itself (brute-force enumeration, scipy's qhull Delaunay and
 * halfspace intersection, closed forms, libm, curand's host Philox, finite
 * differences).  Nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 16
#define OR_NO_ID INT32_MIN

static int32_t face_id(int a, int s) { return -(2 * a + s + 1); }
static int face_axis(int32_t id) { return (-id - 1) >> 1; }
static int face_side(int32_t id) { return (-id - 1) & 1; }

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops from now on (timing at one core). */
void or_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,  */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Ten rounds; each  */
/* round multiplies words 0 and 2 by the two Philox constants and mixes the  */
/* high halves with words 1, 3 and the key; the key is bumped by the Weyl    */
/* constants between rounds.                                                 */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* binary32 log / sin / cos written out from textbook series so that the    */
/* Gaussian draw has one bit-exact definition on every machine:             */
/*  log: m*2^e with m in [sqrt(1/2), sqrt(2)), ln m = 2 artanh((m-1)/(m+1))  */
/*       (series through s^11), e*ln2 split in a high part with trailing     */
/*       zeros and a low part (Cody & Waite style reduction);               */
/*  sin, cos: Taylor series on [0, pi/4] after an exact octant reduction of  */
/*       the 24-bit angle fraction.                                          */
/* Each operation is rounded separately, in the order written.              */
/* ------------------------------------------------------------------------ */
static float f32_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t f32_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

float or_log32(float x) {
  uint32_t b = f32_bits(x);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = f32_from_bits((b & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = m * 0.5f;
    e = e + 1;
  }
  float s = (m - 1.0f) / (m + 1.0f);
  float z = s * s;
  float p = 0x1.745d18p-4f;          /* 1/11 */
  p = p * z; p = p + 0x1.c71c72p-4f;  /* 1/9 */
  p = p * z; p = p + 0x1.24924ap-3f;  /* 1/7 */
  p = p * z; p = p + 0x1.99999ap-3f;  /* 1/5 */
  p = p * z; p = p + 0x1.555556p-2f;  /* 1/3 */
  p = p * z; p = p + 1.0f;
  float lnm = (s + s) * p;
  float fe = (float)e;
  float lo = fe * 0x1.7f7d1cp-20f;    /* ln2 - ln2_hi */
  float hi = fe * 0x1.62e4p-1f;       /* ln2_hi, exact product */
  return hi + (lo + lnm);
}

static float sin_poly(float phi) {
  float z = phi * phi;
  float p = 0x1.71de3ap-19f;           /* 1/9! */
  p = p * z; p = p + -0x1.a01a02p-13f; /* -1/7! */
  p = p * z; p = p + 0x1.111112p-7f;   /* 1/5! */
  p = p * z; p = p + -0x1.555556p-3f;  /* -1/3! */
  p = p * z; p = p + 1.0f;
  return phi * p;
}

static float cos_poly(float phi) {
  float z = phi * phi;
  float p = -0x1.27e4fcp-22f;          /* -1/10! */
  p = p * z; p = p + 0x1.a01a02p-16f;  /* 1/8! */
  p = p * z; p = p + -0x1.6c16c2p-10f; /* -1/6! */
  p = p * z; p = p + 0x1.555556p-5f;   /* 1/4! */
  p = p * z; p = p + -0.5f;            /* -1/2! */
  p = p * z; p = p + 1.0f;
  return p;
}

/* cos and sin of 2*pi*(a24 / 2^24), a24 a 24-bit integer. */
void or_sincos2pi24(uint32_t a24, float* c_out, float* s_out) {
  uint32_t q = a24 >> 21;
  uint32_t f = a24 & 0x1fffffu;
  uint32_t g = (q & 1u) ? (0x200000u - f) : f;
  float phi = 0x1.921fb6p+2f * ((float)g * 0x1p-24f);
  float C = cos_poly(phi), S = sin_poly(phi);
  float c, s;
  switch (q) {
    case 0: c = C;  s = S;  break;
    case 1: c = S;  s = C;  break;
    case 2: c = -S; s = C;  break;
    case 3: c = -C; s = S;  break;
    case 4: c = -C; s = -S; break;
    case 5: c = -S; s = -C; break;
    case 6: c = S;  s = -C; break;
    default: c = C; s = -S; break;
  }
  *c_out = c;
  *s_out = s;
}

/* Box-Muller pair from two 32-bit words: U in (0,1) from the top 23 bits of
 * x0 (odd multiple of 2^-24), angle fraction from the top 24 bits of x1. */
static void box_muller(uint32_t x0, uint32_t x1, float* z0, float* z1) {
  float U = (float)((x0 >> 9) * 2u + 1u) * 0x1p-24f;
  float r = sqrtf(-2.0f * or_log32(U));
  float c, s;
  or_sincos2pi24(x1 >> 8, &c, &s);
  *z0 = r * c;
  *z1 = r * s;
}

/* Uniform direction on S^{d-1} for ray k of cell `cell` of point set `set`
 * (Section 3.1: a normalised standard Gaussian draw).  Philox counter
 * (block, k, cell, set), key (seed low, seed high); each block of four words
 * gives four Gaussians.  The Gaussian is binary32, the normalisation
 * binary64: u = z * (1 / sqrt(sum z^2)). */
void or_mc_direction(uint64_t seed, uint32_t set, uint32_t cell, uint32_t ray, int d, double* u) {
  float z[OR_MAXD + 4];
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int blk = 0; blk * 4 < d; ++blk) {
    uint32_t ctr[4] = {(uint32_t)blk, ray, cell, set}, o[4];
    or_philox4x32_10(ctr, key, o);
    box_muller(o[0], o[1], &z[4 * blk + 0], &z[4 * blk + 1]);
    box_muller(o[2], o[3], &z[4 * blk + 2], &z[4 * blk + 3]);
  }
  double ss = 0.0;
  for (int k = 0; k < d; ++k) {
    double zk = (double)z[k];
    ss = ss + zk * zk;
  }
  double inv = 1.0 / sqrt(ss);
  for (int k = 0; k < d; ++k) u[k] = (double)z[k] * inv;
}

void or_mc_gaussian32(uint64_t seed, uint32_t set, uint32_t cell, uint32_t ray, int d, float* z) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  float tmp[OR_MAXD + 4];
  for (int blk = 0; blk * 4 < d; ++blk) {
    uint32_t ctr[4] = {(uint32_t)blk, ray, cell, set}, o[4];
    or_philox4x32_10(ctr, key, o);
    box_muller(o[0], o[1], &tmp[4 * blk + 0], &tmp[4 * blk + 1]);
    box_muller(o[2], o[3], &tmp[4 * blk + 2], &tmp[4 * blk + 3]);
  }
  for (int k = 0; k < d; ++k) z[k] = tmp[k];
}

/* ------------------------------------------------------------------------ */
/* RayCast (Section 2.2, Eq. (t), Algorithm 1): the exact first bisector    */
/* hit.  The incircle iteration of Algorithm 1 stops exactly at             */
/*   t* = min over nodes j not in eta with den_j = <u, x_j - g> > 0 of     */
/*   t_j = (|x_j - v|^2 - |g - v|^2) / (2 den_j),                           */
/* plus the faces of [0,1]^d, so the oracle evaluates that minimum directly. */
/* Canonical binary64 order: w = x_j - g, p = v - g,                         */
/* num = sum w_k w_k - 2 sum p_k w_k, den = sum u_k w_k (left to right),    */
/* t = num / (2 den); faces t = (b - v_a) / u_a.  Ties: order (t, class, id) */
/* with nodes (class 0, by id) before faces (class 1, by 2a+s).             */
/* ------------------------------------------------------------------------ */
static int in_list(int32_t id, const int32_t* eta, int m) {
  for (int q = 0; q < m; ++q)
    if (eta[q] == id) return 1;
  return 0;
}

static int better(double t, int cls, int64_t key, double bt, int bcls, int64_t bkey) {
  if (t < bt) return 1;
  if (t > bt) return 0;
  if (cls != bcls) return cls < bcls;
  return key < bkey;
}

/* eta: m ids (m >= 1), eta[0] = g must be a node.  Returns hit and t. */
static void raycast1(const double* X, int64_t N, int d, int box, const double* v, const double* u,
                     const int32_t* eta, int m, int32_t* hit, double* tout, int64_t* ties) {
  const double* g = X + (int64_t)eta[0] * d;
  double p[OR_MAXD];
  for (int k = 0; k < d; ++k) p[k] = v[k] - g[k];
  double bt = INFINITY;
  int bcls = 2;
  int64_t bkey = 0;
  int32_t bid = OR_NO_ID;
  for (int64_t j = 0; j < N; ++j) {
    if (in_list((int32_t)j, eta, m)) continue;
    const double* x = X + j * d;
    double w[OR_MAXD];
    for (int k = 0; k < d; ++k) w[k] = x[k] - g[k];
    double den = 0.0;
    for (int k = 0; k < d; ++k) den = den + u[k] * w[k];
    if (!(den > 0.0)) continue;
    double ww = 0.0, pw = 0.0;
    for (int k = 0; k < d; ++k) ww = ww + w[k] * w[k];
    for (int k = 0; k < d; ++k) pw = pw + p[k] * w[k];
    double num = ww - 2.0 * pw;
    double t = num / (2.0 * den);
    if (ties && t == bt && bcls == 0) ++*ties;
    if (better(t, 0, j, bt, bcls, bkey)) {
      bt = t; bcls = 0; bkey = j; bid = (int32_t)j;
    }
  }
  if (box) {
    for (int a = 0; a < d; ++a) {
      int s;
      double b;
      if (u[a] < 0.0) { s = 0; b = 0.0; }
      else if (u[a] > 0.0) { s = 1; b = 1.0; }
      else continue;
      int32_t id = face_id(a, s);
      if (in_list(id, eta, m)) continue;
      double t = (b - v[a]) / u[a];
      if (better(t, 1, 2 * a + s, bt, bcls, bkey)) {
        bt = t; bcls = 1; bkey = 2 * a + s; bid = id;
      }
    }
  }
  *hit = bid;
  *tout = bt;
}

/* Batch of R rays; eta rows have `stride` entries padded with INT32_MIN. */
void or_raycast(const double* X, int64_t N, int d, int box, const double* origins, const double* dirs,
                const int32_t* eta, int stride, int64_t R, int32_t* hit, double* t) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < R; ++r) {
    const int32_t* e = eta + r * stride;
    int m = 0;
    while (m < stride && e[m] != OR_NO_ID) ++m;
    raycast1(X, N, d, box, origins + r * d, dirs + r * d, e, m, &hit[r], &t[r], NULL);
  }
}

/* ------------------------------------------------------------------------ */
/* Monte Carlo volumes and interface areas (Section 3.1, Algorithm 3).      */
/* For ray k of cell i: u_k uniform on the sphere, l_k = t* of the RayCast  */
/* from v = g = x_i with eta = {i}.                                          */
/*   V_i  = S_{d-1} / (d R) * sum_k l_k^d                                    */
/*   A_ij = S_{d-1} / R * sum_{k: hit j} l_k^{d-1} / |n_ij . u_k|            */
/* with n_ij = (x_j - x_i)/|x_j - x_i|; because l = |w|^2 / (2 u.w) for a   */
/* node hit, l^{d-1}/|n.u| = 2 l^d / |w|, the form used here.  A face hit on */
/* axis a has n = e_a and contributes l^{d-1} / |u_a|.                      */
/* l^d is formed by repeated multiplication l*l*...*l (left to right).      */
/* ------------------------------------------------------------------------ */
double or_sphere_area(int d) { /* S_{d-1} = 2 pi^{d/2} / Gamma(d/2) */
  return 2.0 * pow(M_PI, 0.5 * d) / tgamma(0.5 * d);
}

static double ipow(double l, int n) {
  double r = 1.0;
  for (int q = 0; q < n; ++q) r = (q == 0) ? l : r * l;
  return r;
}

/* Raycasts of all N*R MC rays.  hit, l: N*R, ray (i,k) at i*R+k. */
void or_mc_rays(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set, int32_t* hit,
                double* l) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < N; ++i) {
    int32_t eta[1] = {(int32_t)i};
    for (int64_t k = 0; k < R; ++k) {
      double u[OR_MAXD];
      or_mc_direction(seed, set, (uint32_t)i, (uint32_t)k, d, u);
      raycast1(X, N, d, 1, X + i * d, u, eta, 1, &hit[i * R + k], &l[i * R + k], NULL);
    }
  }
}

/* Per-ray area term a_k (before the S_{d-1}/R scale). */
static double area_term(const double* X, int d, int64_t i, int32_t j, double l, const double* u) {
  if (j >= 0) {
    double ww = 0.0;
    for (int k = 0; k < d; ++k) {
      double w = X[(int64_t)j * d + k] - X[i * d + k];
      ww = ww + w * w;
    }
    return (2.0 * ipow(l, d)) / sqrt(ww);
  }
  int a = face_axis(j);
  return ipow(l, d - 1) / fabs(u[a]);
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Row i of the CSR holds the distinct hit ids of cell i, ascending (faces,
 * negative, first).  Returns nnz, or -1 if cap is too small. */
int64_t or_mc_reduce(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set,
                     const int32_t* hit, const double* l, double* V, int64_t* rowptr, int32_t* col, double* A,
                     int64_t cap) {
  const double S = or_sphere_area(d);
  const double cV = S / ((double)d * (double)R), cA = S / (double)R;
  int32_t* ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
  int64_t nnz = 0;
  rowptr[0] = 0;
  for (int64_t i = 0; i < N; ++i) {
    const int32_t* h = hit + i * R;
    const double* li = l + i * R;
    memcpy(ids, h, sizeof(int32_t) * (size_t)R);
    qsort(ids, (size_t)R, sizeof(int32_t), cmp_i32);
    int64_t row0 = nnz;
    for (int64_t k = 0; k < R; ++k) {
      if (k > 0 && ids[k] == ids[k - 1]) continue;
      if (nnz >= cap) { free(ids); return -1; }
      col[nnz] = ids[k];
      A[nnz] = 0.0;
      ++nnz;
    }
    double vs = 0.0;
    for (int64_t k = 0; k < R; ++k) {
      double u[OR_MAXD];
      or_mc_direction(seed, set, (uint32_t)i, (uint32_t)k, d, u);
      vs = vs + ipow(li[k], d);
      int64_t lo = row0, hi = nnz;
      while (hi - lo > 1) { /* binary search for hit id in the row */
        int64_t mid = (lo + hi) / 2;
        if (col[mid] <= h[k]) lo = mid; else hi = mid;
      }
      A[lo] = A[lo] + area_term(X, d, i, h[k], li[k], u);
    }
    V[i] = cV * vs;
    for (int64_t q = row0; q < nnz; ++q) A[q] = cA * A[q];
    rowptr[i + 1] = nnz;
  }
  free(ids);
  return nnz;
}

/* The estimator with the argmins held fixed (the saved hit ids): l_k is
 * recomputed from the same formula as in the RayCast for the saved hit, so
 * this is a smooth function of X that the tests difference numerically. */
static double fixed_l(const double* X, int d, int64_t i, int32_t j, const double* u) {
  const double* xi = X + i * d;
  if (j >= 0) {
    double w[OR_MAXD], den = 0.0, ww = 0.0, pw = 0.0;
    for (int k = 0; k < d; ++k) w[k] = X[(int64_t)j * d + k] - xi[k];
    for (int k = 0; k < d; ++k) den = den + u[k] * w[k];
    for (int k = 0; k < d; ++k) ww = ww + w[k] * w[k];
    (void)pw; /* v = g = x_i, so p = 0 and num = ww exactly */
    return ww / (2.0 * den);
  }
  int a = face_axis(j);
  double b = face_side(j) ? 1.0 : 0.0;
  return (b - xi[a]) / u[a];
}

void or_mc_eval_fixed(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set,
                      const int32_t* hit, const int64_t* rowptr, const int32_t* col, double* V, double* A) {
  const double S = or_sphere_area(d);
  const double cV = S / ((double)d * (double)R), cA = S / (double)R;
  for (int64_t i = 0; i < N; ++i) {
    double vs = 0.0;
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) A[q] = 0.0;
    for (int64_t k = 0; k < R; ++k) {
      double u[OR_MAXD];
      or_mc_direction(seed, set, (uint32_t)i, (uint32_t)k, d, u);
      int32_t j = hit[i * R + k];
      double l = fixed_l(X, d, i, j, u);
      vs = vs + ipow(l, d);
      for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q)
        if (col[q] == j) { A[q] = A[q] + area_term(X, d, i, j, l, u); break; }
    }
    V[i] = cV * vs;
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) A[q] = cA * A[q];
  }
}

/* Adjoint of the MC estimator with directions and argmins fixed (pathwise,
 * quotient rule at each saved argmin).  For a node hit j, w = x_j - x_i,
 * l = |w|^2/(2 u.w):  dl/dw = (w - l u) / (u.w),  dl/dx_j = dl/dw,
 * dl/dx_i = -dl/dw.  Area term a = 2 l^d / |w|:
 *   da/dw = (2 d l^{d-1} / |w|) dl/dw - (2 l^d / |w|^3) w.
 * Face hit on axis a: l = (b - x_ia)/u_a, dl/dx_ia = -1/u_a, a = l^{d-1}/|u_a|,
 *   da/dl = (d-1) l^{d-2} / |u_a|.
 * gX = sum_i gV_i dV_i/dX + sum_ij gA_ij dA_ij/dX. */
void or_mc_adjoint(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set,
                   const int32_t* hit, const double* l, const int64_t* rowptr, const int32_t* col,
                   const double* gV, const double* gA, double* gX) {
  const double S = or_sphere_area(d);
  const double cV = S / ((double)d * (double)R), cA = S / (double)R;
  for (int64_t q = 0; q < N * d; ++q) gX[q] = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    const double* xi = X + i * d;
    for (int64_t k = 0; k < R; ++k) {
      double u[OR_MAXD];
      or_mc_direction(seed, set, (uint32_t)i, (uint32_t)k, d, u);
      int32_t j = hit[i * R + k];
      double lk = l[i * R + k];
      double gAij = 0.0;
      for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q)
        if (col[q] == j) { gAij = gA[q]; break; }
      double ld1 = ipow(lk, d - 1), ld = ipow(lk, d);
      if (j >= 0) {
        const double* xj = X + (int64_t)j * d;
        double w[OR_MAXD], den = 0.0, ww = 0.0;
        for (int k2 = 0; k2 < d; ++k2) w[k2] = xj[k2] - xi[k2];
        for (int k2 = 0; k2 < d; ++k2) den = den + u[k2] * w[k2];
        for (int k2 = 0; k2 < d; ++k2) ww = ww + w[k2] * w[k2];
        double nw = sqrt(ww);
        for (int k2 = 0; k2 < d; ++k2) {
          double dl = (w[k2] - lk * u[k2]) / den;
          double dV = cV * (double)d * ld1 * dl;
          double dA = cA * ((2.0 * (double)d * ld1 / nw) * dl - (2.0 * ld / (nw * nw * nw)) * w[k2]);
          double G = gV[i] * dV + gAij * dA;
          gX[(int64_t)j * d + k2] += G;
          gX[i * d + k2] -= G;
        }
      } else {
        int a = face_axis(j);
        double dl = -1.0 / u[a];
        double dadl = (d >= 2) ? (double)(d - 1) * ipow(lk, d - 2) / fabs(u[a]) : 0.0;
        double G = gV[i] * cV * (double)d * ld1 * dl + gAij * cA * dadl * dl;
        gX[i * d + a] += G;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Monte Carlo integrals of a function f over the cell boundaries and the    */
/* cell volumes (Section 3.1, Eqs. mc-help1 and full_MC_integration,         */
/* Algorithm 3), from the rays of a finished run (directions, hits, l):      */
/*   F_d[i][j] = S_{d-1}/R sum_{k: hit j} f(r_k) a_k,  r_k = x_i + l_k u_k,  */
/*               a_k the area term of A above (so f = 1 gives A exactly);    */
/*   F_V[i]    = S_{d-1}/(R m) sum_k sum_{s<m} f(y_ks) t_ks^{d-1} l_k^d,     */
/*               y_ks = x_i + (t_ks l_k) u_k,  t_ks ~ U(0,1).                */
/* F_V is the polar change of variables around x_i, dV = l^d t^{d-1} dt dS   */
/* over the sphere and t in (0,1), with the normalisation of Algorithm 3:    */
/* the mean of t^{d-1} over uniform t is 1/d, so f = 1 estimates the volume. */
/* t_ks = (w + 1/2) 2^-32 with w word (s mod 4) of Philox4x32-10 at counter  */
/* (2^31 + s div 4, k, cell, set), key (seed low, seed high): counters the   */
/* directions (block < 4) never use.  Sums run over k, then s, in order.     */
/* f (kind, axis, coef = c0, b[0..d), q[0..d)):                              */
/*   kind 0: f = 1;                                                          */
/*   kind 1: f = c0 + sum_a b_a y_a + sum_a q_a y_a^2, left to right, the    */
/*           linear terms first;                                             */
/*   kind 2: f = sin(y_axis^2) (the integrand of the paper's Section 4).    */
/* ------------------------------------------------------------------------ */
double or_func_eval(int kind, int axis, const double* coef, int d, const double* y) {
  if (kind == 1) {
    double s = coef[0];
    for (int a = 0; a < d; ++a) s = s + coef[1 + a] * y[a];
    for (int a = 0; a < d; ++a) s = s + coef[1 + d + a] * (y[a] * y[a]);
    return s;
  }
  if (kind == 2) return sin(y[axis] * y[axis]);
  return 1.0;
}

double or_mc_tsample(uint64_t seed, uint32_t set, uint32_t cell, uint32_t ray, uint32_t s) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {0x80000000u + (s >> 2), ray, cell, set}, o[4];
  or_philox4x32_10(ctr, key, o);
  return ((double)o[s & 3] + 0.5) * 0x1p-32;
}

/* Cells cells[0..ncells): their rays' hit and l in rows of R (hit, l), their  */
/* CSR rows in rowptr (local, rowptr[0] = 0) and col; writes FV[c] and the    */
/* row entries of Fd. */
void or_mc_integrals(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set, int64_t ncells,
                     const int64_t* cells, const int32_t* hit, const double* l, const int64_t* rowptr,
                     const int32_t* col, int kind, int axis, const double* coef, int64_t m, double* FV,
                     double* Fd) {
  (void)N;
  const double S = or_sphere_area(d);
  const double cA = S / (double)R, cV = S / ((double)R * (double)m);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t c = 0; c < ncells; ++c) {
    const int64_t i = cells[c];
    const double* xi = X + i * d;
    const int32_t* h = hit + c * R;
    const double* lc = l + c * R;
    for (int64_t q = rowptr[c]; q < rowptr[c + 1]; ++q) Fd[q] = 0.0;
    double fv = 0.0;
    for (int64_t k = 0; k < R; ++k) {
      double u[OR_MAXD], r[OR_MAXD], y[OR_MAXD];
      or_mc_direction(seed, set, (uint32_t)i, (uint32_t)k, d, u);
      const double lk = lc[k];
      for (int a = 0; a < d; ++a) r[a] = xi[a] + lk * u[a];
      int64_t lo = rowptr[c], hi = rowptr[c + 1];
      while (hi - lo > 1) { /* the hit id's entry in the row */
        int64_t mid = (lo + hi) / 2;
        if (col[mid] <= h[k]) lo = mid; else hi = mid;
      }
      Fd[lo] = Fd[lo] + or_func_eval(kind, axis, coef, d, r) * area_term(X, d, i, h[k], lk, u);
      const double ld = ipow(lk, d);
      for (int64_t s2 = 0; s2 < m; ++s2) {
        const double t = or_mc_tsample(seed, set, (uint32_t)i, (uint32_t)k, (uint32_t)s2);
        const double tl = t * lk;
        for (int a = 0; a < d; ++a) y[a] = xi[a] + tl * u[a];
        const double w = ipow(t, d - 1) * ld;
        fv = fv + or_func_eval(kind, axis, coef, d, y) * w;
      }
    }
    FV[c] = cV * fv;
    for (int64_t q = rowptr[c]; q < rowptr[c + 1]; ++q) Fd[q] = cA * Fd[q];
  }
}

void or_mc_tsamples(uint64_t seed, uint32_t set, int64_t ncells, int64_t R, int64_t m, double* out) {
  for (int64_t i = 0; i < ncells; ++i)
    for (int64_t k = 0; k < R; ++k)
      for (int64_t s = 0; s < m; ++s)
        out[(i * R + k) * m + s] = or_mc_tsample(seed, set, (uint32_t)i, (uint32_t)k, (uint32_t)s);
}

/* ------------------------------------------------------------------------ */
/* Heuristic Monte-Carlo integration (Section 3.3): from interface areas     */
/* A_ij (the CSR of an MC run, or exact ones) and the vertices of the        */
/* diagram (sorted tuples and coordinates, from the traversal):              */
/*   V_i  = (1/d) sum_j h_ij A_ij   (h_ij = |x_j - x_i|/2, or the distance   */
/*          from x_i to the box face j);                                     */
/*   F_ij = (d/(d+1)) (1/K_ij) sum_k f(nu_k) A_ij + (1/(d+1)) f(y_ij) A_ij   */
/*          over the K_ij vertices nu_k whose tuple holds both i and j, and  */
/*          their mean y_ij;                                                 */
/*   I_i  = sum_j (h_ij/d) ((d/(d+1)) F_ij + (1/(d+1)) A_ij f(x_i)), the     */
/*          cone rule of Eq. (leibniz-int) over the pyramid with base facet  */
/*          ij and apex x_i (height h_ij).                                   */
/* Sums over k run in ascending vertex order, sums over j in CSR order.      */
/* F_ij = 0 for an entry with no vertex (K_ij = 0).                          */
/* In binary64: y = (sum nu) / K per axis, mean f = (sum f) / K,             */
/* F = (cd * mean f + c1 * f(y)) * A with cd = d/(d+1), c1 = 1/(d+1);        */
/* I sums (h / d) * (cd * F + c1 * (A * f(x_i))); V = (sum h A) / d.         */
/* ------------------------------------------------------------------------ */
static int64_t find_entry(const int64_t* rowptr, const int32_t* col, int64_t i, int32_t j) {
  int64_t lo = rowptr[i], hi = rowptr[i + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (col[mid] < j) lo = mid + 1; else hi = mid;
  }
  return (lo < rowptr[i + 1] && col[lo] == j) ? lo : -1;
}

void or_hmc(const double* X, int64_t N, int d, const int64_t* rowptr, const int32_t* col, const double* A,
            const int32_t* tuples, const double* coords, int64_t nv, int kind, int axis, const double* coef,
            double* VH, double* FH, double* IH, int64_t* K_out) {
  const int64_t nnz = rowptr[N];
  int64_t* K = (int64_t*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(int64_t));
  double* fs = (double*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
  double* ys = (double*)calloc((size_t)(nnz > 0 ? nnz : 1) * d, sizeof(double));
  const double cd = (double)d / (double)(d + 1), c1 = 1.0 / (double)(d + 1);
  for (int64_t v = 0; v < nv; ++v) {
    const int32_t* sg = tuples + v * (d + 1);
    const double* nu = coords + v * d;
    const double fnu = or_func_eval(kind, axis, coef, d, nu);
    for (int a = 0; a <= d; ++a) {
      if (sg[a] < 0 || sg[a] >= N) continue;
      for (int b = 0; b <= d; ++b) {
        if (b == a) continue;
        const int64_t e = find_entry(rowptr, col, sg[a], sg[b]);
        if (e < 0) continue;
        K[e] += 1;
        fs[e] = fs[e] + fnu;
        for (int c = 0; c < d; ++c) ys[e * d + c] = ys[e * d + c] + nu[c];
      }
    }
  }
  for (int64_t e = 0; e < nnz; ++e) {
    double F = 0.0;
    if (K[e] > 0) {
      double y[OR_MAXD];
      for (int c = 0; c < d; ++c) y[c] = ys[e * d + c] / (double)K[e];
      const double mf = fs[e] / (double)K[e];
      F = (cd * mf + c1 * or_func_eval(kind, axis, coef, d, y)) * A[e];
    }
    if (FH) FH[e] = F;
    fs[e] = F;  /* kept for the cells */
    if (K_out) K_out[e] = K[e];
  }
  for (int64_t i = 0; i < N; ++i) {
    const double* xi = X + i * d;
    const double fxi = or_func_eval(kind, axis, coef, d, xi);
    double vh = 0.0, ih = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = col[e];
      double h;
      if (j >= 0) {
        double ww = 0.0;
        for (int c = 0; c < d; ++c) {
          double w = X[(int64_t)j * d + c] - xi[c];
          ww = ww + w * w;
        }
        h = 0.5 * sqrt(ww);
      } else {
        h = face_side(j) ? 1.0 - xi[face_axis(j)] : xi[face_axis(j)];
      }
      vh = vh + h * A[e];
      ih = ih + (h / (double)d) * (cd * fs[e] + c1 * (A[e] * fxi));
    }
    if (VH) VH[i] = vh / (double)d;
    if (IH) IH[i] = ih;
  }
  free(K);
  free(fs);
  free(ys);
}

/* ------------------------------------------------------------------------ */
/* Exact volumes, interface areas and integrals of the piecewise linear      */
/* interpolant of f (Section 3.2, Algorithms 4-5, IterativeVolume) from the  */
/* vertices of the diagram.  For cell i the faces are walked depth first:    */
/* level 1 is the cell (its vertices: tuples holding i), a face at level D   */
/* keeps the vertices of its parent whose tuple also holds the generator j   */
/* that defines it (candidates j in ascending id, not already in the face),  */
/* down to the edges at level d (exactly two vertices nu, nu').  Each edge   */
/* closes the simplex (x_i, m_2, ..., m_{d-1}, nu, nu') with m_D the mean of */
/* the level-D face's vertices; its volume is |det(m_2 - x_i, ...,           */
/* m_{d-1} - x_i, nu - x_i, nu' - x_i)| / d! (Gaussian elimination with      */
/* partial pivoting, first maximal |entry|).  Integrals follow Algorithm 5:  */
/* an edge returns F = (f(nu) + f(nu'))/2 V; a face at level 1 < D < d       */
/* returns (sum V, ((d-D+1)/(d-D+2)) sum F + (1/(d-D+2)) f(m_D) sum V); the  */
/* cell takes F_i = (d/(d+1)) sum F + (1/(d+1)) f(x_i) sum V.  A facet ij    */
/* (level 2) gives A_ij = V_ij d / h_ij and Fd_ij = F_ij d / h_ij with       */
/* h_ij = |x_j - x_i|/2 or the distance to the box face.  Row i of the CSR   */
/* lists the facets in ascending j.  Returns -1 if an edge does not have     */
/* two vertices (degenerate input) or cap is too small, else nnz.  d >= 2.   */
/* ------------------------------------------------------------------------ */
#define OR_LZ_MAXD 8

static double lz_absdet(double* M, int d) { /* M row-major d x d, destroyed */
  double det = 1.0;
  for (int c = 0; c < d; ++c) {
    int p = c;
    for (int r = c + 1; r < d; ++r)
      if (fabs(M[r * d + c]) > fabs(M[p * d + c])) p = r;
    if (M[p * d + c] == 0.0) return 0.0;
    if (p != c)
      for (int k = 0; k < d; ++k) { double t = M[c * d + k]; M[c * d + k] = M[p * d + k]; M[p * d + k] = t; }
    for (int r = c + 1; r < d; ++r) {
      const double mlt = M[r * d + c] / M[c * d + c];
      for (int k = c + 1; k < d; ++k) M[r * d + k] = M[r * d + k] - mlt * M[c * d + k];
    }
    det = det * M[c * d + c];
  }
  return fabs(det);
}

static int tuple_has(const int32_t* t, int L, int32_t g) {
  for (int q = 0; q < L; ++q) if (t[q] == g) return 1;
  return 0;
}

typedef struct {
  const double* X; int d; int64_t i;
  const int32_t* tuples; const double* coords;
  int kind, axis; const double* coef;
  double fact, mid[OR_LZ_MAXD + 1][OR_LZ_MAXD];
  int32_t S[OR_LZ_MAXD + 2];
  int bad;
} lz_ctx;

/* smallest generator > prev in the tuples of list[0..n) that is not in S[0..D) */
static int64_t lz_next(const lz_ctx* c, const int64_t* list, int64_t n, int D, int64_t prev) {
  int64_t best = INT64_MAX;
  for (int64_t q = 0; q < n; ++q) {
    const int32_t* t = c->tuples + list[q] * (c->d + 1);
    for (int k = 0; k <= c->d; ++k) {
      const int64_t g = t[k];
      if (g <= prev || g >= best) continue;
      int in = 0;
      for (int s2 = 0; s2 < D; ++s2) in |= (c->S[s2] == g);
      if (!in) best = g;
    }
  }
  return best;
}

/* face at level D with vertex list (list, n); returns its V, F */
static void lz_rec(lz_ctx* c, int D, const int64_t* list, int64_t n, double* Vout, double* Fout,
                   double* Afac, double* Ffac, int64_t* nf, int64_t cap) {
  const int d = c->d;
  const double* xi = c->X + c->i * d;
  if (D == d) { /* an edge */
    if (n != 2) { c->bad = 1; *Vout = 0.0; *Fout = 0.0; return; }
    double M[OR_LZ_MAXD * OR_LZ_MAXD];
    for (int col = 0; col < d; ++col) {
      const double* p = col < d - 2 ? c->mid[col + 2] : c->coords + list[col - (d - 2)] * d;
      for (int r = 0; r < d; ++r) M[r * d + col] = p[r] - xi[r];
    }
    const double V = lz_absdet(M, d) / c->fact;
    const double f0 = or_func_eval(c->kind, c->axis, c->coef, d, c->coords + list[0] * d);
    const double f1 = or_func_eval(c->kind, c->axis, c->coef, d, c->coords + list[1] * d);
    *Vout = V;
    *Fout = (0.5 * (f0 + f1)) * V;
    return;
  }
  double fm = 0.0;
  if (D >= 2) { /* the face's vertex mean */
    for (int a = 0; a < d; ++a) c->mid[D][a] = 0.0;
    for (int64_t q = 0; q < n; ++q)
      for (int a = 0; a < d; ++a) c->mid[D][a] = c->mid[D][a] + c->coords[list[q] * d + a];
    for (int a = 0; a < d; ++a) c->mid[D][a] = c->mid[D][a] / (double)n;
    fm = or_func_eval(c->kind, c->axis, c->coef, d, c->mid[D]);
  }
  int64_t* child = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  double sv = 0.0, sf = 0.0;
  int64_t j = INT64_MIN;
  while ((j = lz_next(c, list, n, D, j)) != INT64_MAX) {
    int64_t m = 0;
    for (int64_t q = 0; q < n; ++q)
      if (tuple_has(c->tuples + list[q] * (d + 1), d + 1, (int32_t)j)) child[m++] = list[q];
    c->S[D] = (int32_t)j;
    double v = 0.0, f = 0.0;
    lz_rec(c, D + 1, child, m, &v, &f, Afac, Ffac, nf, cap);
    if (D == 1) { /* facet ij */
      double h;
      if (j >= 0) {
        double ww = 0.0;
        for (int a = 0; a < d; ++a) { double w = c->X[j * d + a] - xi[a]; ww = ww + w * w; }
        h = 0.5 * sqrt(ww);
      } else {
        h = face_side((int32_t)j) ? 1.0 - xi[face_axis((int32_t)j)] : xi[face_axis((int32_t)j)];
      }
      if (*nf < cap) {
        Afac[*nf] = (v * (double)d) / h;
        Ffac[*nf] = (f * (double)d) / h;
      } else {
        c->bad = 1;
      }
      *nf += 1;
    }
    sv = sv + v;
    sf = sf + f;
  }
  free(child);
  *Vout = sv;
  if (D == 1) {
    const double fx = or_func_eval(c->kind, c->axis, c->coef, d, xi);
    *Fout = ((double)d / (double)(d + 1)) * sf + (1.0 / (double)(d + 1)) * fx * sv;
  } else {
    const double w1 = (double)(d - D + 1) / (double)(d - D + 2), w0 = 1.0 / (double)(d - D + 2);
    *Fout = w1 * sf + w0 * fm * sv;
  }
}

int64_t or_leibniz(const double* X, int64_t N, int d, const int32_t* tuples, const double* coords, int64_t nv,
                   int kind, int axis, const double* coef, double* V, double* F, int64_t* rowptr, int32_t* col,
                   double* A, double* Fd, int64_t cap) {
  if (d < 2 || d > OR_LZ_MAXD) return -1;
  /* vertex lists of the cells, ascending vertex order */
  int64_t* cnt = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
  for (int64_t v = 0; v < nv; ++v)
    for (int k = 0; k <= d; ++k) {
      const int32_t g = tuples[v * (d + 1) + k];
      if (g >= 0 && g < N) cnt[g + 1] += 1;
    }
  for (int64_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
  int64_t* lists = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cnt[N] > 0 ? cnt[N] : 1));
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) cur[i] = cnt[i];
  for (int64_t v = 0; v < nv; ++v)
    for (int k = 0; k <= d; ++k) {
      const int32_t g = tuples[v * (d + 1) + k];
      if (g >= 0 && g < N) lists[cur[g]++] = v;
    }
  lz_ctx c;
  memset(&c, 0, sizeof(c));
  c.X = X; c.d = d; c.tuples = tuples; c.coords = coords; c.kind = kind; c.axis = axis; c.coef = coef;
  c.fact = 1.0;
  for (int k = 2; k <= d; ++k) c.fact = c.fact * (double)k;
  int64_t nf = 0;
  rowptr[0] = 0;
  for (int64_t i = 0; i < N; ++i) {
    c.i = i;
    c.S[0] = (int32_t)i;
    const int64_t f0 = nf;
    double v = 0.0, f = 0.0;
    lz_rec(&c, 1, lists + cnt[i], cnt[i + 1] - cnt[i], &v, &f, A, Fd, &nf, cap);
    /* the facet ids of row i, ascending (the order the walk visited them) */
    int64_t j = INT64_MIN, q = f0;
    while ((j = lz_next(&c, lists + cnt[i], cnt[i + 1] - cnt[i], 1, j)) != INT64_MAX) {
      if (q < cap) col[q] = (int32_t)j;
      ++q;
    }
    V[i] = v;
    F[i] = f;
    rowptr[i + 1] = nf;
  }
  free(cnt); free(lists); free(cur);
  return c.bad ? -1 : nf;
}

/* ------------------------------------------------------------------------ */
/* Vertices: Algorithm 2 (VoronoiGraph) with the box faces as generators.   */
/* ------------------------------------------------------------------------ */

/* Coordinates of the vertex with sorted generator tuple sig[0..d] (Section  */
/* 2.1: equidistant to its nodes, on its faces).  With x0 the first node and */
/* y = r - x0: fixed axes y_a = s_a - x0_a; for every other node k,          */
/* 2 w_k . y = |w_k|^2 (w_k = x_k - x0), moved to the free axes; Gaussian    */
/* elimination with partial pivoting (first maximal |pivot|, magnitudes      */
/* compared after rounding to binary32), multipliers and back substitution   */
/* through the rounded reciprocal 1/pivot.  Returns 0 if two faces share an  */
/* axis or the system is singular.                                           */
int or_vertex_coords(const double* X, int d, const int32_t* sig, double* r) {
  int fixed[OR_MAXD], side[OR_MAXD];
  for (int a = 0; a < d; ++a) fixed[a] = 0;
  int nodes[OR_MAXD + 1], m = 0;
  for (int q = 0; q <= d; ++q) {
    if (sig[q] >= 0) { nodes[m++] = sig[q]; continue; }
    int a = face_axis(sig[q]);
    if (fixed[a]) return 0;
    fixed[a] = 1;
    side[a] = face_side(sig[q]);
  }
  if (m < 1) return 0;
  const double* x0 = X + (int64_t)nodes[0] * d;
  int freeax[OR_MAXD], nf = 0;
  double y[OR_MAXD];
  for (int a = 0; a < d; ++a) {
    if (fixed[a]) y[a] = (side[a] ? 1.0 : 0.0) - x0[a];
    else freeax[nf++] = a;
  }
  if (nf != m - 1) return 0;
  double M[OR_MAXD][OR_MAXD], b[OR_MAXD];
  for (int rr = 0; rr < nf; ++rr) {
    const double* xk = X + (int64_t)nodes[rr + 1] * d;
    double w[OR_MAXD], ww = 0.0;
    for (int a = 0; a < d; ++a) w[a] = xk[a] - x0[a];
    for (int a = 0; a < d; ++a) ww = ww + w[a] * w[a];
    for (int a = 0; a < d; ++a)
      if (fixed[a]) ww = ww - (2.0 * w[a]) * y[a];
    for (int c = 0; c < nf; ++c) M[rr][c] = 2.0 * w[freeax[c]];
    b[rr] = ww;
  }
  double inv[OR_MAXD];
  for (int c = 0; c < nf; ++c) {
    int piv = c;
    for (int rr = c + 1; rr < nf; ++rr)
      if ((float)fabs(M[rr][c]) > (float)fabs(M[piv][c])) piv = rr;
    if (M[piv][c] == 0.0) return 0;
    if (piv != c) {
      for (int cc = 0; cc < nf; ++cc) { double tmp = M[c][cc]; M[c][cc] = M[piv][cc]; M[piv][cc] = tmp; }
      double tb = b[c]; b[c] = b[piv]; b[piv] = tb;
    }
    inv[c] = 1.0 / M[c][c];
    for (int rr = c + 1; rr < nf; ++rr) {
      double f = M[rr][c] * inv[c];
      for (int cc = c + 1; cc < nf; ++cc) M[rr][cc] = M[rr][cc] - f * M[c][cc];
      b[rr] = b[rr] - f * b[c];
    }
  }
  double z[OR_MAXD];
  for (int c = nf - 1; c >= 0; --c) {
    double s = b[c];
    for (int cc = c + 1; cc < nf; ++cc) s = s - M[c][cc] * z[cc];
    z[c] = s * inv[c];
  }
  for (int c = 0; c < nf; ++c) y[freeax[c]] = z[c];
  for (int a = 0; a < d; ++a) r[a] = fixed[a] ? (side[a] ? 1.0 : 0.0) : x0[a] + y[a];
  return 1;
}

/* SearchDirection (Algorithm 2): unit u orthogonal to the affine hull of the
 * nodes of eta = sig minus sig[drop] and to the normals of its faces,
 * pointing away from the dropped generator.  The nodes of eta give rows
 * w_k = x_k - g (g its first node) over the axes not fixed by its faces; the
 * null vector is found by Gaussian elimination with complete pivoting (first
 * maximal |entry| in row-major order, magnitudes compared after rounding to
 * binary32; multipliers through the rounded reciprocal 1/pivot), the
 * non-pivot column set to 1, back substitution, then u = z * (1/|z|).
 * Sign: a dropped node e must give
 * u . (x_e - g) < 0 (same sum order as the RayCast's den); a dropped lower
 * face u_a > 0, an upper face u_a < 0.  Returns 0 if eta has no node or the
 * rows are degenerate. */
int or_search_direction(const double* X, int d, const int32_t* sig, int drop, double* u) {
  int32_t eta[OR_MAXD];
  int m = 0;
  for (int q = 0; q <= d; ++q)
    if (q != drop) eta[m++] = sig[q];
  int fixed[OR_MAXD];
  for (int a = 0; a < d; ++a) fixed[a] = 0;
  int nodes[OR_MAXD], mn = 0;
  for (int q = 0; q < d; ++q) {
    if (eta[q] >= 0) nodes[mn++] = eta[q];
    else fixed[face_axis(eta[q])] = 1;
  }
  if (mn < 1) return 0;
  int freeax[OR_MAXD], nf = 0;
  for (int a = 0; a < d; ++a)
    if (!fixed[a]) freeax[nf++] = a;
  if (nf != mn) return 0;
  const double* g = X + (int64_t)nodes[0] * d;
  int nr = mn - 1;
  double M[OR_MAXD][OR_MAXD];
  for (int rr = 0; rr < nr; ++rr) {
    const double* xk = X + (int64_t)nodes[rr + 1] * d;
    for (int c = 0; c < nf; ++c) M[rr][c] = xk[freeax[c]] - g[freeax[c]];
  }
  int colperm[OR_MAXD];
  for (int c = 0; c < nf; ++c) colperm[c] = c;
  double inv[OR_MAXD];
  for (int c = 0; c < nr; ++c) {
    int pr = c, pc = c;
    float best = -1.0f;
    for (int rr = c; rr < nr; ++rr)
      for (int cc = c; cc < nf; ++cc)
        if ((float)fabs(M[rr][cc]) > best) { best = (float)fabs(M[rr][cc]); pr = rr; pc = cc; }
    if (M[pr][pc] == 0.0) return 0;
    if (pr != c)
      for (int cc = 0; cc < nf; ++cc) { double tmp = M[c][cc]; M[c][cc] = M[pr][cc]; M[pr][cc] = tmp; }
    if (pc != c) {
      for (int rr = 0; rr < nr; ++rr) { double tmp = M[rr][c]; M[rr][c] = M[rr][pc]; M[rr][pc] = tmp; }
      int tp = colperm[c]; colperm[c] = colperm[pc]; colperm[pc] = tp;
    }
    inv[c] = 1.0 / M[c][c];
    for (int rr = c + 1; rr < nr; ++rr) {
      double f = M[rr][c] * inv[c];
      for (int cc = c + 1; cc < nf; ++cc) M[rr][cc] = M[rr][cc] - f * M[c][cc];
    }
  }
  /* permuted unknowns zp[0..nf-1]; zp[nf-1] = 1 (the free column) */
  double zp[OR_MAXD];
  zp[nf - 1] = 1.0;
  for (int c = nr - 1; c >= 0; --c) {
    double s = -M[c][nf - 1];
    for (int cc = c + 1; cc < nr; ++cc) s = s - M[c][cc] * zp[cc];
    zp[c] = s * inv[c];
  }
  double z[OR_MAXD];
  for (int c = 0; c < nf; ++c) z[colperm[c]] = zp[c];
  double nz = 0.0;
  for (int c = 0; c < nf; ++c) nz = nz + z[c] * z[c];
  const double invn = 1.0 / sqrt(nz);
  for (int a = 0; a < d; ++a) u[a] = 0.0;
  for (int c = 0; c < nf; ++c) u[freeax[c]] = z[c] * invn;
  int32_t e = sig[drop];
  int flip;
  if (e >= 0) {
    const double* xe = X + (int64_t)e * d;
    double den = 0.0;
    for (int a = 0; a < d; ++a) den = den + u[a] * (xe[a] - g[a]);
    if (den == 0.0) return 0;
    flip = den > 0.0;
  } else {
    int a = face_axis(e);
    if (u[a] == 0.0) return 0;
    flip = face_side(e) ? (u[a] > 0.0) : (u[a] < 0.0);
  }
  if (flip)
    for (int a = 0; a < d; ++a) u[a] = -u[a];
  return 1;
}

/* --- tuple hash set (open addressing, linear probing) ------------------- */
typedef struct {
  int L;            /* tuple length */
  int64_t cap;      /* power of two */
  int64_t count;
  int64_t* slot;    /* -1 empty, else entry index */
  int32_t* keys;    /* entry tuples */
  int32_t* vals;
  int64_t ecap;
} thash;

static uint64_t tuple_hash(const int32_t* t, int L) {
  uint64_t h = 1469598103934665603ull;
  for (int q = 0; q < L; ++q) {
    h ^= (uint32_t)t[q];
    h *= 1099511628211ull;
    h ^= h >> 29;
  }
  return h;
}

static void th_init(thash* h, int L, int64_t cap) {
  h->L = L; h->cap = cap; h->count = 0; h->ecap = cap / 2;
  h->slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
  for (int64_t q = 0; q < cap; ++q) h->slot[q] = -1;
  h->keys = (int32_t*)malloc(sizeof(int32_t) * (size_t)(h->ecap * L));
  h->vals = (int32_t*)malloc(sizeof(int32_t) * (size_t)h->ecap);
}

static void th_free(thash* h) { free(h->slot); free(h->keys); free(h->vals); }

static void th_grow(thash* h) {
  int64_t ncap = h->cap * 2;
  int64_t* ns = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncap);
  for (int64_t q = 0; q < ncap; ++q) ns[q] = -1;
  for (int64_t e = 0; e < h->count; ++e) {
    uint64_t s = tuple_hash(h->keys + e * h->L, h->L) & (uint64_t)(ncap - 1);
    while (ns[s] >= 0) s = (s + 1) & (uint64_t)(ncap - 1);
    ns[s] = e;
  }
  free(h->slot);
  h->slot = ns; h->cap = ncap; h->ecap = ncap / 2;
  h->keys = (int32_t*)realloc(h->keys, sizeof(int32_t) * (size_t)(h->ecap * h->L));
  h->vals = (int32_t*)realloc(h->vals, sizeof(int32_t) * (size_t)h->ecap);
}

/* returns entry index; *created = 1 if inserted (val set to 0) */
static int64_t th_find_or_insert(thash* h, const int32_t* t, int* created) {
  if (h->count + 1 > h->ecap) th_grow(h);
  uint64_t s = tuple_hash(t, h->L) & (uint64_t)(h->cap - 1);
  while (h->slot[s] >= 0) {
    int64_t e = h->slot[s];
    if (memcmp(h->keys + e * h->L, t, sizeof(int32_t) * (size_t)h->L) == 0) { *created = 0; return e; }
    s = (s + 1) & (uint64_t)(h->cap - 1);
  }
  int64_t e = h->count++;
  memcpy(h->keys + e * h->L, t, sizeof(int32_t) * (size_t)h->L);
  h->vals[e] = 0;
  h->slot[s] = e;
  *created = 1;
  return e;
}

static int64_t th_find(const thash* h, const int32_t* t) {
  uint64_t s = tuple_hash(t, h->L) & (uint64_t)(h->cap - 1);
  while (h->slot[s] >= 0) {
    int64_t e = h->slot[s];
    if (memcmp(h->keys + e * h->L, t, sizeof(int32_t) * (size_t)h->L) == 0) return e;
    s = (s + 1) & (uint64_t)(h->cap - 1);
  }
  return -1;
}

static void sort_small(int32_t* t, int L) {
  for (int a = 1; a < L; ++a) {
    int32_t x = t[a];
    int b = a - 1;
    while (b >= 0 && t[b] > x) { t[b + 1] = t[b]; --b; }
    t[b + 1] = x;
  }
}

static int edge_has_node(const int32_t* sig, int d, int drop) {
  for (int q = 0; q <= d; ++q)
    if (q != drop && sig[q] >= 0) return 1;
  return 0;
}

static void edge_of(const int32_t* sig, int d, int drop, int32_t* eta) {
  int m = 0;
  for (int q = 0; q <= d; ++q)
    if (q != drop) eta[m++] = sig[q];
}

/* Descent (Algorithm 2): from node s, cast rays in random directions
 * projected orthogonally to the span of the current generators until d+1
 * generators are found.  Directions come from or_mc_direction on set
 * 0xFFFFFFFF (cell = s, ray = step).  Returns 1 and the sorted tuple. */
int or_descent(const double* X, int64_t N, int d, int32_t s, int32_t* sig_out) {
  int32_t sig[OR_MAXD + 1];
  int m = 1;
  sig[0] = s;
  double r[OR_MAXD];
  for (int a = 0; a < d; ++a) r[a] = X[(int64_t)s * d + a];
  for (int step = 0; m < d + 1; ++step) {
    if (step > 64 * (d + 1)) return 0;
    double u[OR_MAXD];
    or_mc_direction(0x5EEDull, 0xFFFFFFFFu, (uint32_t)s, (uint32_t)step, d, u);
    /* constraint rows: x_k - g for the other nodes, e_a for faces */
    int32_t g = -1;
    for (int q = 0; q < m; ++q)
      if (sig[q] >= 0 && (g < 0 || sig[q] < g)) g = sig[q];
    double B[OR_MAXD + 1][OR_MAXD];
    int nb = 0;
    for (int q = 0; q < m; ++q) {
      if (sig[q] == g) continue;
      if (sig[q] >= 0)
        for (int a = 0; a < d; ++a) B[nb][a] = X[(int64_t)sig[q] * d + a] - X[(int64_t)g * d + a];
      else {
        for (int a = 0; a < d; ++a) B[nb][a] = 0.0;
        B[nb][face_axis(sig[q])] = 1.0;
      }
      ++nb;
    }
    /* modified Gram-Schmidt on the rows, then project u */
    for (int q = 0; q < nb; ++q) {
      for (int q2 = 0; q2 < q; ++q2) {
        double dp = 0.0;
        for (int a = 0; a < d; ++a) dp = dp + B[q][a] * B[q2][a];
        for (int a = 0; a < d; ++a) B[q][a] = B[q][a] - dp * B[q2][a];
      }
      double nn = 0.0;
      for (int a = 0; a < d; ++a) nn = nn + B[q][a] * B[q][a];
      nn = sqrt(nn);
      if (nn == 0.0) return 0;
      for (int a = 0; a < d; ++a) B[q][a] = B[q][a] / nn;
    }
    for (int q = 0; q < nb; ++q) {
      double dp = 0.0;
      for (int a = 0; a < d; ++a) dp = dp + u[a] * B[q][a];
      for (int a = 0; a < d; ++a) u[a] = u[a] - dp * B[q][a];
    }
    for (int a = 0; a < d; ++a) /* a face in sig pins its axis exactly */
      for (int q = 0; q < m; ++q)
        if (sig[q] < 0 && face_axis(sig[q]) == a) u[a] = 0.0;
    double nu = 0.0;
    for (int a = 0; a < d; ++a) nu = nu + u[a] * u[a];
    nu = sqrt(nu);
    if (!(nu > 1e-12)) continue;
    for (int a = 0; a < d; ++a) u[a] = u[a] / nu;
    int32_t eta[OR_MAXD + 1];
    eta[0] = g;
    int me = 1;
    for (int q = 0; q < m; ++q)
      if (sig[q] != g) eta[me++] = sig[q];
    int32_t hit;
    double t;
    raycast1(X, N, d, 1, r, u, eta, me, &hit, &t, NULL);
    if (hit == OR_NO_ID) return 0;
    for (int a = 0; a < d; ++a) r[a] = r[a] + t * u[a];
    sig[m++] = hit;
  }
  sort_small(sig, d + 1);
  for (int q = 0; q <= d; ++q) sig_out[q] = sig[q];
  return 1;
}

/* Exhaustive traversal.  Returns the number of vertices V (tuples V*(d+1) in
 * discovery order, coords V*d), -1 if max_vertices is too small, -2 if the
 * seed fails, -3 on a degenerate direction or coordinate solve.
 * stats[0] = raycasts, stats[1] = rediscoveries (0 expected), stats[2] =
 * exact ties seen. */
int64_t or_vertices(const double* X, int64_t N, int d, int32_t seed_node, int64_t max_vertices,
                    int32_t* tuples, double* coords, int64_t* stats) {
  int L = d + 1;
  thash V, G;
  th_init(&V, L, 1024);
  th_init(&G, d, 1024);
  int64_t raycasts = 0, redisc = 0, ties = 0;
  int32_t sig0[OR_MAXD + 1];
  if (!or_descent(X, N, d, seed_node, sig0)) { th_free(&V); th_free(&G); return -2; }
  int created;
  th_find_or_insert(&V, sig0, &created);
  for (int q = 0; q <= d; ++q) {
    if (!edge_has_node(sig0, d, q)) continue;
    int32_t eta[OR_MAXD];
    edge_of(sig0, d, q, eta);
    int64_t e = th_find_or_insert(&G, eta, &created);
    G.vals[e] += 1;
  }
  int64_t head = 0; /* FIFO queue = entries in insertion order */
  int64_t rc = 0;
  while (head < V.count) {
    int32_t sig[OR_MAXD + 1];
    memcpy(sig, V.keys + head * L, sizeof(int32_t) * (size_t)L);
    ++head;
    double r[OR_MAXD];
    if (!or_vertex_coords(X, d, sig, r)) { rc = -3; break; }
    for (int q = 0; q <= d; ++q) {
      if (!edge_has_node(sig, d, q)) continue;
      int32_t eta[OR_MAXD + 1];
      edge_of(sig, d, q, eta);
      int64_t e = th_find(&G, eta);
      if (e >= 0 && G.vals[e] >= 2) continue;
      double u[OR_MAXD];
      if (!or_search_direction(X, d, sig, q, u)) { rc = -3; break; }
      /* reference generator g = first node of eta (eta is sorted) */
      int32_t er[OR_MAXD + 1];
      int gpos = 0;
      while (eta[gpos] < 0) ++gpos;
      er[0] = eta[gpos];
      int me = 1;
      for (int q2 = 0; q2 < d; ++q2)
        if (q2 != gpos) er[me++] = eta[q2];
      int32_t hit;
      double t;
      raycast1(X, N, d, 1, r, u, er, me, &hit, &t, &ties);
      ++raycasts;
      if (hit == OR_NO_ID) continue; /* unbounded ray: impossible with the box */
      int32_t ns[OR_MAXD + 1];
      for (int q2 = 0; q2 < d; ++q2) ns[q2] = eta[q2];
      ns[d] = hit;
      sort_small(ns, L);
      th_find_or_insert(&V, ns, &created);
      if (!created) { ++redisc; continue; }
      for (int q2 = 0; q2 <= d; ++q2) {
        if (!edge_has_node(ns, d, q2)) continue;
        int32_t eta2[OR_MAXD];
        edge_of(ns, d, q2, eta2);
        int64_t e2 = th_find_or_insert(&G, eta2, &created);
        G.vals[e2] += 1;
      }
    }
    if (rc) break;
  }
  int64_t nv = V.count;
  if (rc == 0 && nv > max_vertices) rc = -1;
  if (rc == 0) {
    for (int64_t v = 0; v < nv; ++v) {
      memcpy(tuples + v * L, V.keys + v * L, sizeof(int32_t) * (size_t)L);
      or_vertex_coords(X, d, V.keys + v * L, coords + v * d);
    }
  }
  if (stats) { stats[0] = raycasts; stats[1] = redisc; stats[2] = ties; }
  th_free(&V);
  th_free(&G);
  return rc ? rc : nv;
}

/* --- batch helpers for the tests ---------------------------------------- */
/* ------------------------------------------------------------------------ */
/* Random walks on the vertex graph (Section 2.3: the random walk that       */
/* approximates the Voronoi graph, with the incircle RayCast).  Walker w    */
/* starts at the vertex with sorted tuple start[w]; at step s it takes one   */
/* of the edges of its vertex that hold a node: with the valid drop indices */
/* a_0 < ... < a_{n-1} it takes a_k, k = (w0 n) >> 32, w0 = word 0 of       */
/* Philox4x32-10 at counter (s, w, 0x57414C4B, 0), key (seed low, seed      */
/* high); it casts the ray along that edge (SearchDirection, RayCast from   */
/* the vertex, reference node first as in Algorithm 2) and moves to the     */
/* far vertex sort(edge + hit), coordinates re-solved.  wid (nullable) gives */
/* each walker's index w in the draw.  path_t: W x S x (d+1), path_x:       */
/* W x S x d.  Returns 0, or -1 after a degenerate step (the walker then    */
/* stays where it was).                                                      */
/* ------------------------------------------------------------------------ */
int or_random_walk(const double* X, int64_t N, int d, const int32_t* start, int64_t W, int64_t S, uint64_t seed,
                   const int64_t* wid, int32_t* path_t, double* path_x) {
  const int L = d + 1;
  int rc = 0;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t w = 0; w < W; ++w) {
    int32_t sig[OR_MAXD + 1];
    double r[OR_MAXD];
    for (int q = 0; q < L; ++q) sig[q] = start[w * L + q];
    if (!or_vertex_coords(X, d, sig, r)) rc = -1;
    for (int64_t s = 0; s < S; ++s) {
      int valid[OR_MAXD + 1], n = 0;
      for (int q = 0; q < L; ++q)
        if (edge_has_node(sig, d, q)) valid[n++] = q;
      int ok = n > 0;
      if (ok) {
        uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(wid ? wid[w] : w), 0x57414C4Bu, 0u}, o[4];
        or_philox4x32_10(ctr, key, o);
        const int drop = valid[(int)(((uint64_t)o[0] * (uint64_t)n) >> 32)];
        int32_t eta[OR_MAXD + 1], er[OR_MAXD + 1];
        edge_of(sig, d, drop, eta);
        double u[OR_MAXD];
        ok = or_search_direction(X, d, sig, drop, u);
        if (ok) {
          int gpos = 0;
          while (eta[gpos] < 0) ++gpos;
          er[0] = eta[gpos];
          int me = 1;
          for (int q2 = 0; q2 < d; ++q2)
            if (q2 != gpos) er[me++] = eta[q2];
          int32_t hit;
          double t;
          raycast1(X, N, d, 1, r, u, er, me, &hit, &t, NULL);
          ok = hit != OR_NO_ID;
          if (ok) {
            int32_t ns[OR_MAXD + 1];
            double x[OR_MAXD];
            for (int q2 = 0; q2 < d; ++q2) ns[q2] = eta[q2];
            ns[d] = hit;
            sort_small(ns, L);
            ok = or_vertex_coords(X, d, ns, x);
            if (ok) {
              for (int q2 = 0; q2 < L; ++q2) sig[q2] = ns[q2];
              for (int a = 0; a < d; ++a) r[a] = x[a];
            }
          }
        }
      }
      if (!ok) rc = -1;
      for (int q = 0; q < L; ++q) path_t[(w * S + s) * L + q] = sig[q];
      for (int a = 0; a < d; ++a) path_x[(w * S + s) * d + a] = r[a];
    }
  }
  return rc;
}

void or_log32_batch(const float* x, float* y, int64_t n) {
  for (int64_t q = 0; q < n; ++q) y[q] = or_log32(x[q]);
}

void or_sincos2pi24_batch(const uint32_t* a, float* c, float* s, int64_t n) {
  for (int64_t q = 0; q < n; ++q) or_sincos2pi24(a[q] & 0xffffffu, &c[q], &s[q]);
}

void or_philox_batch(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  for (int64_t q = 0; q < n; ++q) or_philox4x32_10(ctr + 4 * q, key, out + 4 * q);
}

/* directions of rays k = 0..R-1 of cells 0..N-1: out[(i*R+k)*d + a] */
void or_mc_directions(uint64_t seed, uint32_t set, int64_t cell0, int64_t N, int64_t R, int d, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i)
    for (int64_t k = 0; k < R; ++k)
      or_mc_direction(seed, set, (uint32_t)(cell0 + i), (uint32_t)k, d, out + (i * R + k) * d);
}

void or_mc_gaussians32(uint64_t seed, uint32_t set, int64_t N, int64_t R, int d, float* out) {
  for (int64_t i = 0; i < N; ++i)
    for (int64_t k = 0; k < R; ++k) or_mc_gaussian32(seed, set, (uint32_t)i, (uint32_t)k, d, out + (i * R + k) * d);
}
