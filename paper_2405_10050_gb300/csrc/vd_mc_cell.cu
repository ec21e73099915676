// vd_mc_cell.cu -- cell-centric Monte Carlo RayCast (Section 3.1,
// Algorithm 3): all R rays of cell i start at x_i with eta = {i}, so they
// share one candidate list.  A thread block takes a cell, stages its list in
// shared memory once (offsets w = x_j - x_i rounded from binary64, their
// binary32 squared lengths and per-candidate error bounds), and then every
// thread casts its own rays through that list:
//   screening  t_j <= T possible iff ww_lo <= 2 T (den + E_den)   (binary32)
//   early exit the list is sorted by distance from x_i; once a candidate is
//              farther than the ball of the current bound can reach inside
//              the node box, every later one is too;
//   recheck    t_j = |w|^2 / (2 u.w) in binary64, canonical order, for the
//              survivors (about one per ray), plus the box faces.
// Rays the list cannot certify go to the generic tree walk.  The batched
// variant runs the cells of many point sets in one persistent launch.
#include <algorithm>
#include <cmath>

#include "vd_ray_common.cuh"

namespace vd {

namespace {

constexpr int kCellThreads = 128;
constexpr int kCellBuf = 4;  // candidates kept per ray (more: the tree walk finishes the ray)

// Shared memory of one cell: offsets [D][K], bounds, ids; per-thread
// candidate buffers; for the recheck each thread's binary64 direction, the
// results of its candidates and each warp's list of (ray, candidate) pairs.
__host__ __device__ inline size_t cell_smem(int D, int K, int threads) {
  return (size_t)K * (D + 5) * 4 + (size_t)threads * kCellBuf * 8 + 8 + (size_t)threads * D * 8 +
         (size_t)threads * kCellBuf * 12;
}

// All R rays of cell i (see the file comment).  Rays the list cannot
// certify are appended to (fb_cell, fb_ray) for the tree walk.
template <int D, int TH>
__device__ void cell_item(const TreeView& tr, int64_t i, int64_t R, uint64_t seed, uint32_t set, int32_t* hit_out,
                          double* t_out, float* smem, Counters* ctr, int32_t* fb_cell, int32_t* fb_ray,
                          int64_t fb_cap, unsigned long long& n_pairs, unsigned long long& n_rech,
                          unsigned long long& n_brute, unsigned long long* fb_count, double* u_out) {
  const int K = tr.K;
  const int d = tr.d;
  float* sw = smem;                      // [D][K] binary32 offsets
  float* snlo = sw + D * K;              // lower bound of |w|^2
  float* snhi = snlo + K;                // upper bound of |w|^2
  float* swn = snhi + K;                 // upper bound of |w|
  float* sflo = swn + K;                 // lower bound of |x_j - x_i|^2 in list order
  int32_t* sid = reinterpret_cast<int32_t*>(sflo + K);
  int32_t* bid = sid + K;                // [TH][kCellBuf]
  float* btl = reinterpret_cast<float*>(bid + TH * kCellBuf);
  double* su64 = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(btl + TH * kCellBuf) + 7) & ~(uintptr_t)7);
  double* bres = su64 + TH * D;          // [TH][kCellBuf] binary64 t of each candidate
  int* wpairs = reinterpret_cast<int*>(bres + TH * kCellBuf);  // [TH / 32][32 * kCellBuf]
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  double* su = su64 + tid * D;
  int* wpair = wpairs + (tid >> 5) * 32 * kCellBuf;
  const float B = tr.coord_abs;
  const float gam = (float)(D + 1) * kU32 * 1.01f;
  const float EW = 4.01f * kU32 * B;
  const float a1 = 1.1f * (gam + 2.1f * kU32);  // |den32 - den| <= a1 |w32|
  const float e1 = 1.1f * (gam + 2.1f * kU32);  // |ww32 - |w|^2| <= e1 ww32
  int32_t* cb = bid + tid * kCellBuf;
  float* ct = btl + tid * kCellBuf;
  const int n = tr.kcnt[i];
  double g64[D];
  float g32[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    g64[k] = k < d ? tr.X[i * d + k] : 0.0;
    g32[k] = k < d ? tr.X32[i * d + k] : 0.f;
  }
  for (int c = tid; c < n; c += TH) {
    const int32_t id = tr.knn[i * K + c];
    float ww = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float w = k < d ? __double2float_rn(tr.X[(int64_t)id * d + k] - g64[k]) : 0.f;
      sw[k * K + c] = w;
      ww = fmaf(w, w, ww);
    }
    snlo[c] = ww * (1.f - e1);
    snhi[c] = ww * (1.f + e1);
    swn[c] = sqrtf(ww) * (1.f + gam);
    sflo[c] = true_d2_lower(ww32_of<D>(tr.X32 + (int64_t)id * d, 1, g32, d), gam, EW, D);
    sid[c] = id;
  }
  const float cert_lo = true_d2_lower(tr.kcert[i], gam, EW, D);
  __syncthreads();
  // every thread runs the same rounds (one ray each, k = k0 + tid), so that
  // the warps can recheck their rays' survivors together
  for (int64_t k0 = 0; k0 < R; k0 += TH) {
    const int64_t k = k0 + tid;
    const bool valid = k < R;
    double u64[D];
#pragma unroll
    for (int q = 0; q < D; ++q) u64[q] = 0.0;
    if (valid) mc_direction<D>(seed, set, (uint32_t)i, (uint32_t)k, d, u64);
    if (u_out && valid) {
#pragma unroll
      for (int q = 0; q < D; ++q)
        if (q < d) u_out[(i * R + k) * d + q] = u64[q];
    }
#pragma unroll
    for (int q = 0; q < D; ++q) su[q] = u64[q];
    float u32[D], p0[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
      u32[q] = __double2float_rn(u64[q]);
      p0[q] = 0.f;
    }
    // box faces: binary32 interval of (b - x_ia) / u_a; a face is kept only
    // if its lower bound does not exceed the smallest upper bound of all
    float T = INFINITY;
    int nc = 0;
    bool overflow = false;
    float ftlo[D];
    int fside[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      ftlo[a] = INFINITY;
      fside[a] = 0;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if (a >= d || !valid) continue;
      float ua = 0.f, va = 0.f;
#pragma unroll
      for (int q = 0; q < D; ++q)
        if (q == a) {
          ua = u32[q];
          va = g32[q];
        }
      // u32 is u64 rounded to nearest, so it has u64's sign; and a component
      // of an MC direction is either 0 or above 5e-12 in magnitude (Box-Muller
      // radius >= 3.4e-4, sine and cosine 0 or >= 3.7e-7, |z| <= 24), so u32
      // is zero exactly when u64 is: both tests run in binary32
      if (ua == 0.f) continue;
      const int s = ua > 0.f ? 1 : 0;
      const float nf = (s ? 1.f : 0.f) - va;
      const float nfs = s ? nf : -nf;
      const float ef = 1.01f * kU32 * (fabsf(va) + fabsf(nf)) + 1e-38f;
      const float au = fabsf(ua);
      const float lo_n = nfs - ef, hi_n = nfs + ef;
      const float tlo = lo_n >= 0.f ? lo_n / (au * (1.f + 2.f * kU32)) * (1.f - 4.f * kU32)
                                    : lo_n / (au * (1.f - 2.f * kU32)) * (1.f + 4.f * kU32);
      const float thi = hi_n >= 0.f ? hi_n / (au * (1.f - 2.f * kU32)) * (1.f + 4.f * kU32)
                                    : hi_n / (au * (1.f + 2.f * kU32)) * (1.f - 4.f * kU32);
      T = fminf(T, thi);
      ftlo[a] = tlo;
      fside[a] = s;
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (ftlo[a] <= T) {
        if (nc < kCellBuf) {
          cb[nc] = face_id(a, fside[a]);
          ct[nc] = ftlo[a];
          ++nc;
        } else {
          overflow = true;  // the tree walk finishes the ray
        }
      }
    Ball<D> ball;
    make_ball<D>(g32, p0, u32, T, B, ball);
    float far2 = far_radius2<D>(tr, ball, g32);
    bool certified = !valid;
    int c = 0;
    for (; c < n && valid; ++c) {
      if (sflo[c] >= far2) {
        certified = true;
        break;
      }
      float den = 0.f;
#pragma unroll
      for (int q = 0; q < D; ++q) den = fmaf(u32[q], sw[q * K + c], den);
      const float e = a1 * swn[c];
      const float dh = den + e;
      const float nlo = snlo[c];
      if (!(dh > 0.f) || nlo > 2.f * T * dh * (1.f + 8.f * kU32)) continue;
      const float dl = den - e;
      const float thi = dl > 0.f ? __fdiv_rn(snhi[c], 2.f * dl) * (1.f + 4.f * kU32) : INFINITY;
      const float tlo = __fdiv_rn(nlo, 2.f * dh) * (1.f - 4.f * kU32);
      if (thi < T) {
        T = thi;
        make_ball<D>(g32, p0, u32, T, B, ball);
        far2 = far_radius2<D>(tr, ball, g32);
      }
      if (tlo <= T && !overflow) {
        if (nc == kCellBuf) {  // drop entries the new bound has excluded
          int m = 0;
          for (int q = 0; q < kCellBuf; ++q)
            if (ct[q] <= T) {
              cb[m] = cb[q];
              ct[m] = ct[q];
              ++m;
            }
          nc = m;
        }
        if (nc < kCellBuf) {
          cb[nc] = sid[c];
          ct[nc] = tlo;
          ++nc;
        } else {
          overflow = true;
        }
      }
    }
    n_pairs += (unsigned long long)c;
    if (!certified) certified = cert_lo >= far2;
    const bool recheck = valid && certified && !overflow;
    if (valid && !recheck) {  // the tree walk finishes the ray, from the bound found so far
      const unsigned long long q = atomicAdd(fb_count, 1ull);
      if ((int64_t)q < fb_cap) {
        fb_cell[q] = (int32_t)i;
        fb_ray[q] = (int32_t)k;
      } else {
        atomicOr(&ctr->flags, kFlagQueue);
      }
      t_out[i * R + k] = (double)T;
    }
    // ---- binary64 recheck of the warp's survivors, one (ray, candidate)
    // pair per lane, canonical order; each ray then takes the best of its own
    int m = 0;
    if (recheck)
      for (int q = 0; q < nc; ++q)
        if (ct[q] <= T) cb[m++] = cb[q];
    int excl = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, excl, o);
      if (lane >= o) excl += y;
    }
    const int total = __shfl_sync(kFull, excl, 31);
    excl -= m;
    for (int q = 0; q < m; ++q) wpair[excl + q] = (lane << 8) | q;
    __syncwarp();
    for (int p = lane; p < total; p += 32) {
      const int owner = wpair[p] >> 8, q = wpair[p] & 255;
      const int ot = (tid & ~31) + owner;  // the owner's thread in the block
      const int32_t id = bid[ot * kCellBuf + q];
      const double* uo = su64 + (int64_t)ot * D;
      double t = NAN;  // NaN: not a candidate (u.w <= 0)
      if (id >= 0) {
        double w[D], den = 0.0, ww = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) w[a] = a < d ? __dadd_rn(tr.X[(int64_t)id * d + a], -g64[a]) : 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a)
          if (a < d) den = __dadd_rn(den, __dmul_rn(uo[a], w[a]));
        if (den > 0.0) {
#pragma unroll
          for (int a = 0; a < D; ++a)
            if (a < d) ww = __dadd_rn(ww, __dmul_rn(w[a], w[a]));
          t = __ddiv_rn(ww, __dmul_rn(2.0, den));  // num = ww since v = g
        }
      } else {
        const int a = face_axis(id), s = face_side(id);
        double ua = 0.0, va = 0.0;
#pragma unroll
        for (int q2 = 0; q2 < D; ++q2)
          if (q2 == a) {
            ua = uo[q2];
            va = g64[q2];
          }
        t = __ddiv_rn(__dadd_rn(s ? 1.0 : 0.0, -va), ua);
      }
      bres[ot * kCellBuf + q] = t;
    }
    n_rech += (lane == 0) ? (unsigned long long)total : 0ull;
    __syncwarp();
    if (recheck) {
      double bt = INFINITY;
      int bc = 2, bk = 0;
      for (int q = 0; q < m; ++q) {
        const double t = bres[tid * kCellBuf + q];
        if (t != t) continue;  // u.w <= 0
        const int32_t id = cb[q];
        const int cls = id >= 0 ? 0 : 1;
        const int key = id >= 0 ? id : 2 * face_axis(id) + face_side(id);
        if (better(t, cls, key, bt, bc, bk)) {
          bt = t;
          bc = cls;
          bk = key;
        }
      }
      hit_out[i * R + k] = gen_from_key(bc, bk);
      t_out[i * R + k] = bt;
    }
    __syncwarp();  // the next round rewrites the pair list and the results
  }
  __syncthreads();
}

// Shared memory of one cell on the binary64 path: offsets [D][K] and |w|^2
// in binary64, distance bounds and ids.
__host__ __device__ inline size_t cell_smem_f64(int D, int K) { return (size_t)K * (8 * D + 16); }

// All R rays of cell i with every pair in binary64 (VD_FP64): the same list,
// order and exit test as cell_item, each candidate's t_j = |w|^2 / (2 u.w)
// in the canonical order (w, |w|^2 and u.w summed left to right), the box
// faces in binary64.  The division is skipped when the binary64 product
// shows t_j above the current best by more than the rounding of t_j.
template <int D, int TH>
__device__ void cell_item_f64(const TreeView& tr, int64_t i, int64_t R, uint64_t seed, uint32_t set,
                              int32_t* hit_out, double* t_out, double* smem, Counters* ctr, int32_t* fb_cell,
                              int32_t* fb_ray, int64_t fb_cap, unsigned long long& n_pairs,
                              unsigned long long* fb_count, double* u_out) {
  const int K = tr.K;
  const int d = tr.d;
  double* sw = smem;                                 // [D][K] w = x_j - x_i
  double* sww = sw + D * K;                          // |w|^2
  float* sflo = reinterpret_cast<float*>(sww + K);   // lower bound of |x_j - x_i|^2 in list order
  int32_t* sid = reinterpret_cast<int32_t*>(sflo + K);
  const int tid = threadIdx.x;
  const float B = tr.coord_abs;
  const float gam = (float)(D + 1) * kU32 * 1.01f;
  const float EW = 4.01f * kU32 * B;
  const int n = tr.kcnt[i];
  double g64[D];
  float g32[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    g64[k] = k < d ? tr.X[i * d + k] : 0.0;
    g32[k] = k < d ? tr.X32[i * d + k] : 0.f;
  }
  for (int c = tid; c < n; c += TH) {
    const int32_t id = tr.knn[i * K + c];
    double ww = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double w = k < d ? __dadd_rn(tr.X[(int64_t)id * d + k], -g64[k]) : 0.0;
      sw[k * K + c] = w;
      if (k < d) ww = __dadd_rn(ww, __dmul_rn(w, w));
    }
    sww[c] = ww;
    sflo[c] = true_d2_lower(ww32_of<D>(tr.X32 + (int64_t)id * d, 1, g32, d), gam, EW, D);
    sid[c] = id;
  }
  const float cert_lo = true_d2_lower(tr.kcert[i], gam, EW, D);
  __syncthreads();
  for (int64_t k = tid; k < R; k += TH) {
    double u64[D];
    mc_direction<D>(seed, set, (uint32_t)i, (uint32_t)k, d, u64);
    if (u_out) {
#pragma unroll
      for (int q = 0; q < D; ++q)
        if (q < d) u_out[(i * R + k) * d + q] = u64[q];
    }
    float u32[D], p0[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
      u32[q] = __double2float_rn(u64[q]);
      p0[q] = 0.f;
    }
    double bt = INFINITY;
    int bc = 2, bk = 0;
    for (int a = 0; a < d; ++a) {  // box faces, t = (b - x_ia) / u_a
      double ua = 0.0, va = 0.0;
#pragma unroll
      for (int q = 0; q < D; ++q)
        if (q == a) {
          ua = u64[q];
          va = g64[q];
        }
      if (ua == 0.0) continue;
      const int sd = ua > 0.0 ? 1 : 0;
      const double t = __ddiv_rn(__dadd_rn(sd ? 1.0 : 0.0, -va), ua);
      if (better(t, 1, 2 * a + sd, bt, bc, bk)) {
        bt = t;
        bc = 1;
        bk = 2 * a + sd;
      }
    }
    // reach of the ball of the current best (binary32, rounded up)
    auto reach = [&]() {
      Ball<D> ball;
      make_ball<D>(g32, p0, u32, f32_up(bt), B, ball);
      return far_radius2<D>(tr, ball, g32);
    };
    float far2 = reach();
    bool certified = false;
    int c = 0;
    for (; c < n; ++c) {
      if (sflo[c] >= far2) {  // this and every later candidate lie outside the ball
        certified = true;
        break;
      }
      double den = 0.0;
#pragma unroll
      for (int q = 0; q < D; ++q)
        if (q < d) den = __dadd_rn(den, __dmul_rn(u64[q], sw[q * K + c]));
      if (!(den > 0.0)) continue;
      const double ww = sww[c];
      // ww > 2 den bt (1 + 2^-50), evaluated with two roundings, implies
      // ww / (2 den) > bt (1 + 2^-51): the rounded t_j exceeds bt
      if (bt < INFINITY && ww > __dmul_rn(__dmul_rn(__dmul_rn(2.0, den), bt), 1.0 + 0x1p-50)) continue;
      const double t = __ddiv_rn(ww, __dmul_rn(2.0, den));  // num = |w|^2 since v = g
      if (better(t, 0, sid[c], bt, bc, bk)) {
        bt = t;
        bc = 0;
        bk = sid[c];
        far2 = reach();
      }
    }
    n_pairs += (unsigned long long)c;
    if (!certified) certified = cert_lo >= far2;
    if (!certified) {  // the binary64 tree walk finishes the ray
      const unsigned long long q = atomicAdd(fb_count, 1ull);
      if ((int64_t)q < fb_cap) {
        fb_cell[q] = (int32_t)i;
        fb_ray[q] = (int32_t)k;
      } else {
        atomicOr(&ctr->flags, kFlagQueue);
      }
      t_out[i * R + k] = bt;
      continue;
    }
    hit_out[i * R + k] = gen_from_key(bc, bk);
    t_out[i * R + k] = bt;
  }
  __syncthreads();
}

template <int TH>
__device__ __forceinline__ void flush_counters(Counters* ctr, unsigned long long n_pairs, unsigned long long n_rech,
                                               unsigned long long n_brute) {
  for (int o = 16; o; o >>= 1) {
    n_pairs += __shfl_xor_sync(kFull, n_pairs, o);
    n_rech += __shfl_xor_sync(kFull, n_rech, o);
    n_brute += __shfl_xor_sync(kFull, n_brute, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&ctr->pairs, n_pairs);
    atomicAdd(&ctr->rechecked, n_rech);
    if (n_brute) atomicAdd(&ctr->aux0, n_brute);
  }
}

// 8 blocks per SM for d <= 5 (64 registers, no spills), no bound above.
template <int D, bool F64>
__global__ void __launch_bounds__(kCellThreads, D <= 5 ? 8 : 1)
    k_mc_cell(TreeView tr, int64_t R, uint64_t seed, uint32_t set, RayOut ro, Counters* ctr, unsigned long long* work,
              int32_t* fb_cell, int32_t* fb_ray, int64_t fb_cap) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int64_t s_cell;
  unsigned long long n_pairs = 0, n_rech = 0, n_brute = 0;
  while (true) {
    if (threadIdx.x == 0) s_cell = (int64_t)atomicAdd(work, 1ull);
    __syncthreads();
    const int64_t i = s_cell;
    __syncthreads();
    if (i >= tr.N) break;
    if constexpr (F64)
      cell_item_f64<D, kCellThreads>(tr, i, R, seed, set, ro.hit, ro.t, reinterpret_cast<double*>(smem), ctr,
                                     fb_cell, fb_ray, fb_cap, n_pairs, &ctr->fallback, ro.u);
    else
      cell_item<D, kCellThreads>(tr, i, R, seed, set, ro.hit, ro.t, smem, ctr, fb_cell, fb_ray, fb_cap, n_pairs,
                                 n_rech, n_brute, &ctr->fallback, ro.u);
  }
  flush_counters<kCellThreads>(ctr, n_pairs, n_rech, n_brute);
}

// Batched: one persistent launch over every cell of every set; the item's
// set is found by binary search over the sets' first items, the dimension
// selects the instantiation.
template <int TH>
__global__ void __launch_bounds__(TH) k_mc_cell_batch(const SetDesc* sets, int nsets, int64_t nitems, int64_t R,
                                                       uint64_t seed, Counters* ctr, unsigned long long* work) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int64_t s_item;
  unsigned long long n_pairs = 0, n_rech = 0, n_brute = 0;
  while (true) {
    if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(work, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    __syncthreads();
    if (item >= nitems) break;
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (sets[mid].item0 <= item) lo = mid;
      else hi = mid - 1;
    }
    const SetDesc& S = sets[lo];
    const int64_t i = item - S.item0;
    switch (S.tv.d) {
#define VD_CASE(DD)                                                                                              \
  case DD:                                                                                                       \
    cell_item<DD, TH>(S.tv, i, R, seed, S.set, S.hit, S.l, smem, ctr, S.fb_cell, S.fb_ray, S.fb_cap,      \
                             n_pairs, n_rech, n_brute, &S.ctr->fallback, nullptr);                               \
    break;
      VD_CASE(1)
      VD_CASE(2)
      VD_CASE(3)
      VD_CASE(4)
      VD_CASE(5)
      VD_CASE(6)
      default:
        cell_item<8, TH>(S.tv, i, R, seed, S.set, S.hit, S.l, smem, ctr, S.fb_cell, S.fb_ray, S.fb_cap,
                                n_pairs, n_rech, n_brute, &S.ctr->fallback, nullptr);
        break;
#undef VD_CASE
    }
  }
  flush_counters<TH>(ctr, n_pairs, n_rech, n_brute);
}

template <int D, bool F64>
cudaError_t launch_cell_d(const TreeView& tv, int64_t R, uint64_t seed, uint32_t set, const RayOut& ro,
                          Counters* ctr, unsigned long long* work, int32_t* fb_cell, int32_t* fb_ray,
                          int64_t fb_cap, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t sm = F64 ? cell_smem_f64(D, tv.K) : cell_smem(D, tv.K, kCellThreads);
  allow_max_dyn_smem(k_mc_cell<D, F64>);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mc_cell<D, F64>, kCellThreads, sm);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(occ, 1), tv.N));
  cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
  k_mc_cell<D, F64><<<(unsigned)grid, kCellThreads, sm, st>>>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray,
                                                              fb_cap);
  count_launch();
  return cudaGetLastError();
}

template <int TH>
cudaError_t launch_batch_th(const SetDesc* sets, int nsets, int64_t nitems, int maxK, int64_t R, uint64_t seed,
                            Counters* ctr, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t sm = cell_smem(8, maxK, TH);
  allow_max_dyn_smem(k_mc_cell_batch<TH>);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mc_cell_batch<TH>, TH, sm);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(occ, 1), nitems));
  unsigned long long* work = reinterpret_cast<unsigned long long*>(&ctr->aux1);
  cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
  k_mc_cell_batch<TH><<<(unsigned)grid, TH, sm, st>>>(sets, nsets, nitems, R, seed, ctr, work);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

// Casts all N*R MC rays of the node set with the cell kernel (lists needed;
// binary32 screening, or every pair in binary64 for VD_FP64); rays it cannot
// certify are finished by the generic kernels on the same precision.
cudaError_t launch_mc_cells(const TreeView& tv, int64_t R, uint64_t seed, uint32_t set, const RayOut& ro,
                            int precision, Counters* ctr, cudaStream_t st, int64_t* nfallback) {
  unsigned long long* work = reinterpret_cast<unsigned long long*>(&ctr->aux1);
  int32_t* fb_cell = ro.fallback_list;
  int32_t* fb_ray = ro.fallback_list + ro.fallback_cap / 2;
  const int64_t fb_cap = ro.fallback_cap / 2;
  cudaMemsetAsync(&ctr->fallback, 0, sizeof(unsigned long long), st);
  cudaError_t e;
  const bool f64 = precision == VD_FP64;
#define VD_CELL(DD)                                                                                  \
  (f64 ? launch_cell_d<DD, true>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, st)      \
       : launch_cell_d<DD, false>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, st))
  switch (tv.d) {
    case 1: e = VD_CELL(1); break;
    case 2: e = VD_CELL(2); break;
    case 3: e = VD_CELL(3); break;
    case 4: e = VD_CELL(4); break;
    case 5: e = VD_CELL(5); break;
    case 6: e = VD_CELL(6); break;
    default: e = VD_CELL(8); break;
  }
#undef VD_CELL
  if (e != cudaSuccess) return e;
  unsigned long long nfb = 0;
  cudaMemcpyAsync(&nfb, &ctr->fallback, sizeof(nfb), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  const int64_t n = std::min<int64_t>((int64_t)nfb, fb_cap);
  if (nfallback) *nfallback += n;
  if (n == 0) return cudaSuccess;
  // the generic kernels finish them: (cell, ray) lists, tree walk
  RaySource rs;
  rs.mode = 1;
  rs.R = n;
  rs.mc_cell = fb_cell;
  rs.mc_ray = fb_ray;
  rs.mc_rpc = R;
  rs.seed = seed;
  rs.set = set;
  rs.box = 1;
  rs.t_hint = 1;
  RayOut r2 = ro;
  r2.fallback_list = nullptr;  // tree walk directly
  r2.fallback_cap = 0;
  TreeView tv2 = tv;
  tv2.K = 0;
  return launch_raycast(tv2, rs, r2, precision, ctr, st, nullptr);
}

cudaError_t mc_batch_reduce(const SetDesc* sets_dev, int nsets, int64_t nitems, int maxd, int64_t R, uint64_t seed,
                            cudaStream_t st);

cudaError_t launch_mc_batch(const SetDesc* sets_dev, const SetDesc* sets_host, int nsets, int64_t nitems, int maxd,
                            int maxK, int64_t R, uint64_t seed, int threads, Counters* ctr, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(sets_host[0].ctr, 0, sizeof(Counters) * nsets, st);
  if (e != cudaSuccess) return e;
  if (threads <= 64) e = launch_batch_th<64>(sets_dev, nsets, nitems, maxK, R, seed, ctr, st);
  else if (threads <= 128) e = launch_batch_th<128>(sets_dev, nsets, nitems, maxK, R, seed, ctr, st);
  else e = launch_batch_th<256>(sets_dev, nsets, nitems, maxK, R, seed, ctr, st);
  if (e != cudaSuccess) return e;
  // rays the lists could not certify: tree walk per set, counts read on the
  // device (a set without such rays costs two empty launches)
  for (int s = 0; s < nsets && e == cudaSuccess; ++s) e = launch_mc_fallback_dev(sets_host[s], R, seed, st);
  if (e != cudaSuccess) return e;
  return mc_batch_reduce(sets_dev, nsets, nitems, maxd, R, seed, st);
}

// The persistent cell kernel alone over the first `nitems` cells of the
// batch (the autotuner's timing run; the rays it writes are written again by
// the full pass).
cudaError_t launch_mc_batch_cells(const SetDesc* sets_dev, const SetDesc* sets_host, int nsets, int64_t nitems,
                                  int maxK, int64_t R, uint64_t seed, int threads, Counters* ctr, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(sets_host[0].ctr, 0, sizeof(Counters) * nsets, st);
  if (e != cudaSuccess) return e;
  if (threads <= 64) return launch_batch_th<64>(sets_dev, nsets, nitems, maxK, R, seed, ctr, st);
  if (threads <= 128) return launch_batch_th<128>(sets_dev, nsets, nitems, maxK, R, seed, ctr, st);
  return launch_batch_th<256>(sets_dev, nsets, nitems, maxK, R, seed, ctr, st);
}

void mc_batch_dims(int threads, int maxd, int maxK, size_t* smem) { *smem = cell_smem(8, maxK, threads); }

}  // namespace vd
