// vd_mc.cu -- Monte Carlo cell volumes and interface areas (Section 3.1,
// Algorithm 3) from the saved per-ray argmins, and their adjoint.
//
// For ray k of cell i with length l_k = t* and hit generator j:
//   V_i  = S_{d-1} / (d R) sum_k l_k^d
//   A_ij = S_{d-1} / R sum_{k: hit j} a_k,
//   a_k  = l^{d-1} / |n_ij . u_k| = 2 l^d / |x_j - x_i|   (node hit, since
//          l = |w|^2 / (2 u.w) with w = x_j - x_i)
//   a_k  = l^{d-1} / |u_a|                               (face on axis a)
// The reductions are deterministic: a warp owns a cell, visits the distinct
// hit ids of the row in ascending order and sums each one's terms with a
// fixed lane-strided order and butterfly.  When the row has few rays per hit
// id (nnz > R / 8, e.g. high d), the warp instead computes the terms of 32
// rays at a time, one per lane, and adds them to their entries in ascending
// ray order (lanes split the components of the adjoint's vectors); which of
// the two orders a row uses depends only on (nnz, R).
//
// Adjoint (directions and argmins held fixed): for a node hit
//   dl/dx_j = (w - l u) / (u.w) = -dl/dx_i,
//   da/dw   = (2 d l^{d-1} / |w|) dl/dw - (2 l^d / |w|^3) w;
// for a face hit dl/dx_ia = -1/u_a, da/dl = (d-1) l^{d-2} / |u_a|.
// Per (i, j) the row pass sums the ray contributions P_ij; x_i receives
// -sum_j P_ij (plus its face terms) and x_j receives sum_i P_ij through a
// column pass over the transposed entries, again in a fixed order.
#include <algorithm>
#include <cmath>

#include "vd_dev.cuh"

namespace vd {

cudaError_t radix_sort_u64(uint64_t* keys, int32_t* vals, uint64_t* ktmp, int32_t* vtmp, int64_t n,
                           uint32_t* counts, unsigned long long* orand, cudaStream_t st);

namespace {

__device__ __forceinline__ double ipow_d(double l, int n) {
  double r = 1.0;
  for (int q = 0; q < n; ++q) r = (q == 0) ? l : __dmul_rn(r, l);
  return r;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// smallest hit id of the row that is > prev (INT_MAX if none)
__device__ __forceinline__ int32_t next_id(const int32_t* h, int64_t R, int32_t prev, bool first, int lane) {
  int32_t best = INT32_MAX;
  for (int64_t k = lane; k < R; k += 32) {
    const int32_t x = h[k];
    if ((first || x > prev) && x < best) best = x;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o));
  return best;
}

// Direction of ray k of cell i: read from the forward pass's copy U (row
// i R + k, d values) when it was kept, else drawn again (the same bits).
template <int D>
__device__ __forceinline__ void ray_dir(const double* U, uint64_t seed, uint32_t set, int64_t i, int64_t k, int64_t R,
                                        int d, double (&u)[D]) {
  if (U) {
    const double* p = U + (i * R + k) * d;
#pragma unroll
    for (int c = 0; c < D; ++c) u[c] = c < d ? p[c] : 0.0;
  } else {
    mc_direction<D>(seed, set, (uint32_t)i, (uint32_t)k, d, u);
  }
}

// position of hit id in the row's ascending ids col[q0 .. q0 + n)
__device__ __forceinline__ int64_t entry_of(const int32_t* col, int64_t q0, int64_t n, int32_t id) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (col[q0 + mid] < id) lo = mid + 1;
    else hi = mid;
  }
  return q0 + lo;
}

// rows with nnz * kFewRays > R take the ray-parallel order
constexpr int kFewRays = 8;

template <int D>
__device__ __forceinline__ double node_area_term(const double* X, int d, int64_t i, int32_t j, double ld) {
  double ww = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (k < d) {
      const double w = __dadd_rn(X[(int64_t)j * d + k], -X[i * d + k]);
      ww = __dadd_rn(ww, __dmul_rn(w, w));
    }
  return __ddiv_rn(__dmul_rn(2.0, ld), __dsqrt_rn(ww));
}

__global__ void k_mc_count(const int32_t* hit, int64_t N, int64_t R, int64_t* nnz) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  const int32_t* h = hit + i * R;
  int64_t n = 0;
  int32_t prev = 0;
  bool first = true;
  while (true) {
    const int32_t id = next_id(h, R, prev, first, lane);
    if (id == INT32_MAX) break;
    ++n;
    prev = id;
    first = false;
  }
  if (lane == 0) nnz[i] = n;
}

// exclusive scan of n int64 values into out[0..n] (single block)
__global__ void k_scan64(const int64_t* in, int64_t n, int64_t* out) {
  __shared__ int64_t part[1024];
  const int64_t seg = (n + 1023) / 1024;
  const int64_t b = threadIdx.x * seg, e = min(n, b + seg);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += in[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int64_t i = b; i < e; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (threadIdx.x == 1023) out[n] = part[1023];
}

constexpr int kMcWarps = 4;      // warps (cells in flight) per block
constexpr int kMcList = 1024;    // matching-ray indices gathered per pass

// Gathers, in ascending ray order from *k0, up to CAP indices k with
// h[k] == id into L; returns their number and advances *k0.  All lanes take
// part, so the binary64 work on the gathered rays runs on full warps.
template <int CAP = kMcList>
__device__ __forceinline__ int gather_rays(const int32_t* h, int64_t R, int32_t id, int64_t* k0, int32_t* L,
                                           int lane) {
  const unsigned lt = (1u << lane) - 1u;
  int m = 0;
  int64_t k = *k0;
  while (k < R && m + 32 <= CAP) {
    const int64_t kk = k + lane;
    const bool match = kk < R && h[kk] == id;
    const unsigned mask = __ballot_sync(kFull, match);
    if (match) L[m + __popc(mask & lt)] = (int32_t)kk;
    m += __popc(mask);
    k += 32;
  }
  __syncwarp();
  *k0 = k;
  return m;
}

// ---- rows sorted by entry (rows with many rays per hit id) ----
// The warp sorts each chunk of up to CH rays of its row by entry
// (stable: ascending ray order within an entry).  Each lane then sums a
// contiguous range of the sorted node rays, one run per entry; runs that
// cross a lane boundary are joined by a segmented scan over the lanes.  The
// binary64 work thus runs on full warps with one pass over the row, and the
// order of every sum depends only on the row's hits.
constexpr int kEnt = kMcList / kFewRays;  // entries of a row on this path
// The adjoint rows sort chunks of half the size: their per-entry sums are
// D + 1 wide, and the smaller sort arrays let 4 blocks share an SM at d <= 4
// (3 with chunks of kMcList).
constexpr int kAdjList = kMcList / 2;

template <int NV, int CH = kMcList>
struct RowScratch {
  static constexpr int kCh = CH;
  double acc[kEnt][NV];  // per-entry sums over the chunks so far
  int32_t Ej[CH];        // entry << 16 | rank within the entry, per ray of the chunk
                         // (the gathered ray indices on the one-pass-per-id path)
  int32_t col[kEnt];     // the row's hit ids, ascending
  int16_t L[CH];         // ray offset (in the chunk) of each sorted position
  int16_t cnt[kEnt];     // rays of the chunk per entry
  int16_t st[kEnt];      // first sorted position per entry
  uint8_t Es[CH];        // entry of each sorted position
};

// Sorts rays k0 .. k0 + C - 1 of the row (hits h, nnz <= kEnt entries in
// S.col) by entry: S.L, S.Es, S.cnt, S.st.
template <int NV, int CH>
__device__ void sort_chunk(const int32_t* h, int64_t k0, int C, int nnz, RowScratch<NV, CH>& S, int lane) {
  for (int e = lane; e < nnz; e += 32) S.cnt[e] = 0;
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  for (int j0 = 0; j0 < C; j0 += 32) {
    const int j = j0 + lane;
    const bool valid = j < C;
    int e = -1;
    if (valid) {
      const int32_t id = h[k0 + j];
      int lo = 0, hi = nnz - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (S.col[mid] < id) lo = mid + 1;
        else hi = mid;
      }
      e = lo;
    }
    const unsigned peers = __match_any_sync(kFull, e);
    const int pre = valid ? S.cnt[e] : 0;
    __syncwarp();
    if (valid) {
      if (lane == __ffs(peers) - 1) S.cnt[e] = (int16_t)(pre + __popc(peers));
      S.Ej[j] = (e << 16) | (pre + __popc(peers & lt));
    }
    __syncwarp();
  }
  // exclusive scan of the counts (kEnt = 4 x 32)
  int loc[kEnt / 32], s = 0;
#pragma unroll
  for (int t = 0; t < kEnt / 32; ++t) {
    const int e = lane * (kEnt / 32) + t;
    loc[t] = e < nnz ? S.cnt[e] : 0;
    s += loc[t];
  }
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  int run = incl - s;
#pragma unroll
  for (int t = 0; t < kEnt / 32; ++t) {
    const int e = lane * (kEnt / 32) + t;
    if (e < nnz) S.st[e] = (int16_t)run;
    run += loc[t];
  }
  __syncwarp();
  for (int j = lane; j < C; j += 32) {
    const int v = S.Ej[j];
    const int e = v >> 16, p = S.st[e] + (v & 0xFFFF);
    S.L[p] = (int16_t)j;
    S.Es[p] = (uint8_t)e;
  }
  __syncwarp();
}

template <int NV, int NR>
__device__ __forceinline__ void put_acc(double (&a)[NV], const double (&r)[NR], bool first) {
#pragma unroll
  for (int v = 0; v < NR; ++v) a[v] = first ? r[v] : __dadd_rn(a[v], r[v]);
}

// Sums the sorted positions F0 .. C - 1 (node rays) per entry into
// S.acc[e][0 .. NR); step(run, reset, e, j) adds ray offset j of entry e to
// run (restarting it when reset).  first: the chunk is the row's first.
template <int NV, int NR, int CH, class Step>
__device__ __forceinline__ void seg_sums(RowScratch<NV, CH>& S, int F0, int C, bool first, int lane, Step step) {
  const int M = C - F0;
  if (M <= 0) return;
  const int Sz = (M + 31) >> 5;
  const int beg = F0 + lane * Sz, end = min(beg + Sz, C);
  double run[NR], hv[NR];
#pragma unroll
  for (int v = 0; v < NR; ++v) run[v] = hv[v] = 0.0;
  int cur = -1, he = -1;
  bool open = false;
  for (int jj = 0; jj < Sz; ++jj) {
    const int p = beg + jj;
    if (p < end) {
      const int e = S.Es[p];
      step(run, e != cur, e, S.L[p]);
      cur = e;
      const int s0 = S.st[e];
      open = p != s0 + S.cnt[e] - 1;
      if (!open) {
        if (s0 >= beg) {  // the entry's rays of this chunk lie in this lane's range
          put_acc<NV, NR>(S.acc[e], run, first);
        } else {  // it began in an earlier lane: joined after the scan
          he = e;
#pragma unroll
          for (int v = 0; v < NR; ++v) hv[v] = run[v];
        }
      }
    }
  }
  // segmented inclusive scan of the open runs at the range ends
  const int key = open ? cur : -2 - lane;
  double tv[NR];
#pragma unroll
  for (int v = 0; v < NR; ++v) tv[v] = open ? run[v] : 0.0;
  const int kp = __shfl_up_sync(kFull, key, 1);
  int f = (lane == 0 || kp != key) ? 1 : 0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int fu = __shfl_up_sync(kFull, f, o);
#pragma unroll
    for (int v = 0; v < NR; ++v) {
      const double up = __shfl_up_sync(kFull, tv[v], o);
      if (lane >= o && !f) tv[v] = __dadd_rn(up, tv[v]);
    }
    if (lane >= o) f |= fu;
  }
  // a run that ended in this lane after beginning in an earlier one: the
  // previous lane's scan value holds the earlier part
#pragma unroll
  for (int v = 0; v < NR; ++v) {
    const double c = __shfl_up_sync(kFull, tv[v], 1);
    if (he >= 0) hv[v] = __dadd_rn(c, hv[v]);
  }
  if (he >= 0) put_acc<NV, NR>(S.acc[he], hv, first);
  __syncwarp();
}

// Area term of ray k of cell i that hit id.
template <int D>
__device__ __forceinline__ double area_term(const double* X, int d, int64_t i, int64_t k, int32_t id, double lk,
                                            uint64_t seed, uint32_t set, const double* U, int64_t R) {
  if (id >= 0) return node_area_term<D>(X, d, i, id, ipow_d(lk, d));
  double u[D];
  ray_dir<D>(U, seed, set, i, k, R, d, u);
  const int a = face_axis(id);
  double ua = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c)
    if (c == a) ua = u[c];
  return __ddiv_rn(ipow_d(lk, d - 1), fabs(ua));
}

template <int D>
__device__ void fill_item(const double* X, int d, int64_t i, int64_t R, uint64_t seed, uint32_t set,
                          const int32_t* hit, const double* l, const int64_t* rowptr, double cV, double cA, double* V,
                          int32_t* col, double* A, RowScratch<2>& S, int lane, const double* U = nullptr) {
  const int32_t* h = hit + i * R;
  const double* li = l + i * R;
  int64_t q = rowptr[i];
  int32_t prev = 0;
  bool first = true;
  const int64_t q0 = q, nnz = rowptr[i + 1] - q0;
  if (nnz * kFewRays <= R && nnz <= kEnt) {
    // rows sorted by entry: V and the node areas from the per-entry sums of l^d
    for (int e = 0;; ++e) {
      const int32_t id = next_id(h, R, prev, first, lane);
      if (id == INT32_MAX) break;
      if (lane == 0) S.col[e] = id;
      prev = id;
      first = false;
    }
    __syncwarp();
    int nfe = 0;  // face entries (negative ids) come first
    for (int e0 = 0; e0 < nnz; e0 += 32) nfe += __popc(__ballot_sync(kFull, e0 + lane < nnz && S.col[e0 + lane] < 0));
    for (int e = lane; e < nnz; e += 32) col[q0 + e] = S.col[e];
    for (int64_t k0 = 0; k0 < R; k0 += kMcList) {
      const int C = R - k0 < kMcList ? (int)(R - k0) : kMcList;
      const bool fst = k0 == 0;
      sort_chunk<2>(h, k0, C, (int)nnz, S, lane);
      if (fst)
        for (int e = lane; e < nnz; e += 32) S.acc[e][0] = S.acc[e][1] = 0.0;
      __syncwarp();
      for (int e = 0; e < nfe; ++e) {  // face entries: l^d and the area terms, a warp per entry
        const int s0 = S.st[e], n = S.cnt[e];
        if (n == 0) continue;
        double r[2] = {0.0, 0.0};
        for (int p = s0 + lane; p < s0 + n; p += 32) {
          const int64_t k = k0 + S.L[p];
          r[0] = __dadd_rn(r[0], ipow_d(li[k], d));
          r[1] = __dadd_rn(r[1], area_term<D>(X, d, i, k, S.col[e], li[k], seed, set, U, R));
        }
        r[0] = warp_sum_d(r[0]);
        r[1] = warp_sum_d(r[1]);
        if (lane == 0) put_acc<2, 2>(S.acc[e], r, fst);
      }
      __syncwarp();
      const int F0 = nfe < nnz ? S.st[nfe] : C;
      seg_sums<2, 1>(S, F0, C, fst, lane, [&](double (&run)[1], bool reset, int, int j) {
        run[0] = __dadd_rn(reset ? 0.0 : run[0], ipow_d(li[k0 + j], d));
      });
    }
    double vs = 0.0;
    for (int e = lane; e < nnz; e += 32) {
      const int32_t id = S.col[e];
      const double s = S.acc[e][0];
      vs = __dadd_rn(vs, s);
      // node hit: the factor 2 / |x_j - x_i| is applied once per entry
      A[q0 + e] = __dmul_rn(cA, id >= 0 ? node_area_term<D>(X, d, i, id, s) : S.acc[e][1]);
    }
    vs = warp_sum_d(vs);
    if (lane == 0) V[i] = __dmul_rn(cV, vs);
    return;
  }
  double vs = 0.0;
  for (int64_t k = lane; k < R; k += 32) vs = __dadd_rn(vs, ipow_d(li[k], d));
  vs = warp_sum_d(vs);
  if (lane == 0) V[i] = __dmul_rn(cV, vs);
  if (nnz * kFewRays > R) {  // few rays per id: terms ray-parallel, sums in ascending ray order
    double* Ts = &S.acc[0][0];
    int32_t* Es = S.Ej;
    while (true) {
      const int32_t id = next_id(h, R, prev, first, lane);
      if (id == INT32_MAX) break;
      if (lane == 0) {
        col[q] = id;
        A[q] = 0.0;
      }
      ++q;
      prev = id;
      first = false;
    }
    __syncwarp();
    for (int64_t k0 = 0; k0 < R; k0 += 32) {
      const int64_t k = k0 + lane;
      if (k < R) {
        const int32_t id = h[k];
        Es[lane] = (int32_t)(entry_of(col, q0, nnz, id) - q0);
        Ts[lane] = area_term<D>(X, d, i, k, id, li[k], seed, set, U, R);
      }
      __syncwarp();
      if (lane == 0)
        for (int r = 0; r < 32 && k0 + r < R; ++r) A[q0 + Es[r]] = __dadd_rn(A[q0 + Es[r]], Ts[r]);
      __syncwarp();
    }
    for (int64_t e = q0 + lane; e < q0 + nnz; e += 32) A[e] = __dmul_rn(cA, A[e]);
    return;
  }
  // more entries than the sorted path holds: one pass over the row per id
  int32_t* L = S.Ej;
  while (true) {
    const int32_t id = next_id(h, R, prev, first, lane);
    if (id == INT32_MAX) break;
    double s = 0.0;
    int64_t k0 = 0;
    while (k0 < R) {
      const int m = gather_rays(h, R, id, &k0, L, lane);
      for (int p = lane; p < m; p += 32) {
        const int32_t k = L[p];
        // node hit: the factor 2 / |x_j - x_i| is applied once per id below
        s = __dadd_rn(s, id >= 0 ? ipow_d(li[k], d) : area_term<D>(X, d, i, k, id, li[k], seed, set, U, R));
      }
      __syncwarp();
    }
    s = warp_sum_d(s);
    if (id >= 0) s = node_area_term<D>(X, d, i, id, s);
    if (lane == 0) {
      col[q] = id;
      A[q] = __dmul_rn(cA, s);
    }
    ++q;
    prev = id;
    first = false;
  }
}

template <int D>
__global__ void __launch_bounds__(kMcWarps * 32, D <= 8 ? 5 : 1)
    k_mc_fill(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set, const int32_t* hit,
              const double* l, const int64_t* rowptr, double cV, double cA, double* V, int32_t* col, double* A,
              const double* U) {
  extern __shared__ __align__(16) unsigned char row_smem[];
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  RowScratch<2>& S = reinterpret_cast<RowScratch<2>*>(row_smem)[threadIdx.x >> 5];
  fill_item<D>(X, d, i, R, seed, set, hit, l, rowptr, cV, cA, V, col, A, S, lane, U);
}

// ---- function integrals F_d, F_V (Algorithm 3's F and F_V) ----
// f at y in binary64, in the operation order include/vd.h states.
template <int D>
__device__ __forceinline__ double func_at(const vd_func& f, int d, const double (&y)[D]) {
  if (f.kind == VD_F_POLY2) {
    double s = f.c0;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (a < d) s = __dadd_rn(s, __dmul_rn(f.b[a], y[a]));
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (a < d) s = __dadd_rn(s, __dmul_rn(f.q[a], __dmul_rn(y[a], y[a])));
    return s;
  }
  if (f.kind == VD_F_SIN_SQ) {
    double ya = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (a == f.axis) ya = y[a];
    return sin(__dmul_rn(ya, ya));
  }
  return 1.0;
}

// y = x_i + s u (per component, product then sum)
template <int D>
__device__ __forceinline__ void ray_point(const double* X, int d, int64_t i, double s, const double (&u)[D],
                                          double (&y)[D]) {
#pragma unroll
  for (int a = 0; a < D; ++a) y[a] = a < d ? __dadd_rn(X[i * d + a], __dmul_rn(s, u[a])) : 0.0;
}

// l^{d-1} / |u_a| of a ray that hit the face id (the area term of a face hit)
template <int D>
__device__ __forceinline__ double face_term(double lk, int d, int32_t id, const double (&u)[D]) {
  const int a = face_axis(id);
  double ua = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c)
    if (c == a) ua = u[c];
  return __ddiv_rn(ipow_d(lk, d - 1), fabs(ua));
}

// One warp per cell.  F_V: lanes take rays k = lane, lane + 32, ..., each
// its m samples in order (four t per Philox call), then a butterfly.  F_d:
// the two orders of the area fill above with each ray's term multiplied by
// f at its hit point, so f = 1 reproduces A bit for bit.
template <int D>
__global__ void __launch_bounds__(kMcWarps * 32) k_mc_func(const double* X, int64_t N, int d, int64_t R,
                                                           uint64_t seed, uint32_t set, const int32_t* hit,
                                                           const double* l, const int64_t* rowptr,
                                                           const int32_t* col, const double* U, vd_func f,
                                                           int64_t m, double cV, double cA, double* FV, double* Fd) {
  extern __shared__ __align__(16) unsigned char row_smem[];
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  RowScratch<1>& S = reinterpret_cast<RowScratch<1>*>(row_smem)[threadIdx.x >> 5];
  const int32_t* h = hit + i * R;
  const double* li = l + i * R;
  if (FV) {
    double fv = 0.0;
    for (int64_t k = lane; k < R; k += 32) {
      double u[D], y[D];
      ray_dir<D>(U, seed, set, i, k, R, d, u);
      const double lk = li[k];
      const double ld = ipow_d(lk, d);
      for (int64_t s0 = 0; s0 < m; s0 += 4) {
        uint32_t c[4] = {0x80000000u + (uint32_t)(s0 >> 2), (uint32_t)k, (uint32_t)i, set};
        philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (s0 + q >= m) break;
          const double t = __dmul_rn(__dadd_rn((double)c[q], 0.5), 0x1p-32);  // (w + 1/2) 2^-32, exact
          ray_point<D>(X, d, i, __dmul_rn(t, lk), u, y);
          fv = __dadd_rn(fv, __dmul_rn(func_at<D>(f, d, y), __dmul_rn(ipow_d(t, d - 1), ld)));
        }
      }
    }
    fv = warp_sum_d(fv);
    if (lane == 0) FV[i] = __dmul_rn(cV, fv);
  }
  if (!Fd) return;
  const int64_t q0 = rowptr[i], nnz = rowptr[i + 1] - q0;
  if (nnz * kFewRays > R) {  // few rays per id: terms ray-parallel, sums in ascending ray order
    double* Ts = &S.acc[0][0];
    int32_t* Es = S.Ej;
    for (int64_t e = q0 + lane; e < q0 + nnz; e += 32) Fd[e] = 0.0;
    __syncwarp();
    for (int64_t k0 = 0; k0 < R; k0 += 32) {
      const int64_t k = k0 + lane;
      if (k < R) {
        const int32_t id = h[k];
        double u[D], r[D];
        ray_dir<D>(U, seed, set, i, k, R, d, u);
        ray_point<D>(X, d, i, li[k], u, r);
        const double a = id >= 0 ? node_area_term<D>(X, d, i, id, ipow_d(li[k], d)) : face_term<D>(li[k], d, id, u);
        Es[lane] = (int32_t)(entry_of(col, q0, nnz, id) - q0);
        Ts[lane] = __dmul_rn(func_at<D>(f, d, r), a);
      }
      __syncwarp();
      if (lane == 0)
        for (int r2 = 0; r2 < 32 && k0 + r2 < R; ++r2) Fd[q0 + Es[r2]] = __dadd_rn(Fd[q0 + Es[r2]], Ts[r2]);
      __syncwarp();
    }
    for (int64_t e = q0 + lane; e < q0 + nnz; e += 32) Fd[e] = __dmul_rn(cA, Fd[e]);
    return;
  }
  if (nnz <= kEnt) {  // rows sorted by entry, the sums of the fill with f's factor on every ray
    for (int e = lane; e < nnz; e += 32) S.col[e] = col[q0 + e];
    __syncwarp();
    int nfe = 0;
    for (int e0 = 0; e0 < nnz; e0 += 32) nfe += __popc(__ballot_sync(kFull, e0 + lane < nnz && S.col[e0 + lane] < 0));
    for (int64_t k0 = 0; k0 < R; k0 += kMcList) {
      const int C = R - k0 < kMcList ? (int)(R - k0) : kMcList;
      const bool fst = k0 == 0;
      sort_chunk<1>(h, k0, C, (int)nnz, S, lane);
      if (fst)
        for (int e = lane; e < nnz; e += 32) S.acc[e][0] = 0.0;
      __syncwarp();
      for (int e = 0; e < nfe; ++e) {
        const int s0 = S.st[e], n = S.cnt[e];
        if (n == 0) continue;
        double r[1] = {0.0};
        for (int p = s0 + lane; p < s0 + n; p += 32) {
          const int64_t k = k0 + S.L[p];
          double u[D], y[D];
          ray_dir<D>(U, seed, set, i, k, R, d, u);
          ray_point<D>(X, d, i, li[k], u, y);
          r[0] = __dadd_rn(r[0], __dmul_rn(func_at<D>(f, d, y), face_term<D>(li[k], d, S.col[e], u)));
        }
        r[0] = warp_sum_d(r[0]);
        if (lane == 0) put_acc<1, 1>(S.acc[e], r, fst);
      }
      __syncwarp();
      const int F0 = nfe < nnz ? S.st[nfe] : C;
      seg_sums<1, 1>(S, F0, C, fst, lane, [&](double (&run)[1], bool reset, int, int j) {
        const int64_t k = k0 + j;
        double u[D], y[D];
        ray_dir<D>(U, seed, set, i, k, R, d, u);
        ray_point<D>(X, d, i, li[k], u, y);
        run[0] = __dadd_rn(reset ? 0.0 : run[0], __dmul_rn(func_at<D>(f, d, y), ipow_d(li[k], d)));
      });
    }
    for (int e = lane; e < nnz; e += 32) {
      const int32_t id = S.col[e];
      const double s = S.acc[e][0];
      Fd[q0 + e] = __dmul_rn(cA, id >= 0 ? node_area_term<D>(X, d, i, id, s) : s);
    }
    return;
  }
  for (int64_t e = q0; e < q0 + nnz; ++e) {
    const int32_t id = col[e];
    double s = 0.0;
    int64_t k0 = 0;
    while (k0 < R) {
      const int mm = gather_rays(h, R, id, &k0, S.Ej, lane);
      for (int p = lane; p < mm; p += 32) {
        const int32_t k = S.Ej[p];
        double u[D], r[D];
        ray_dir<D>(U, seed, set, i, k, R, d, u);
        ray_point<D>(X, d, i, li[k], u, r);
        // node hit: the factor 2 / |x_j - x_i| is applied once per id below
        const double a = id >= 0 ? ipow_d(li[k], d) : face_term<D>(li[k], d, id, u);
        s = __dadd_rn(s, __dmul_rn(func_at<D>(f, d, r), a));
      }
      __syncwarp();
    }
    s = warp_sum_d(s);
    if (id >= 0) s = node_area_term<D>(X, d, i, id, s);
    if (lane == 0) Fd[e] = __dmul_rn(cA, s);
  }
}

// ---- batched reduction over many sets (items = all cells of all sets) ----
__device__ __forceinline__ int find_set(const SetDesc* sets, int nsets, int64_t item) {
  int lo = 0, hi = nsets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (sets[mid].item0 <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_mc_count_batch(const SetDesc* sets, int nsets, int64_t nitems, int64_t R) {
  const int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= nitems) return;
  const SetDesc& S = sets[find_set(sets, nsets, item)];
  const int64_t i = item - S.item0;
  const int32_t* h = S.hit + i * R;
  int64_t n = 0;
  int32_t prev = 0;
  bool first = true;
  while (true) {
    const int32_t id = next_id(h, R, prev, first, lane);
    if (id == INT32_MAX) break;
    ++n;
    prev = id;
    first = false;
  }
  if (lane == 0) S.cnt[i] = n;
}

// one block per set: rowptr = exclusive scan of the set's counts
__global__ void k_scan_batch(const SetDesc* sets) {
  const SetDesc& S = sets[blockIdx.x];
  const int64_t n = S.tv.N;
  __shared__ int64_t part[1024];
  const int64_t seg = (n + 1023) / 1024;
  const int64_t b = threadIdx.x * seg, e = min(n, b + seg);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += S.cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int64_t i = b; i < e; ++i) {
    S.rowptr[i] = run;
    run += S.cnt[i];
  }
  if (threadIdx.x == 1023) S.rowptr[n] = part[1023];
}

__global__ void __launch_bounds__(kMcWarps * 32) k_mc_fill_batch(const SetDesc* sets, int nsets, int64_t nitems,
                                                                 int64_t R, uint64_t seed) {
  extern __shared__ __align__(16) unsigned char row_smem[];
  const int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= nitems) return;
  const SetDesc& SD = sets[find_set(sets, nsets, item)];
  const int64_t i = item - SD.item0;
  RowScratch<2>& S = reinterpret_cast<RowScratch<2>*>(row_smem)[threadIdx.x >> 5];
  switch (SD.tv.d) {
#define VD_FILL(DD)                                                                                              \
  case DD:                                                                                                       \
    fill_item<DD>(SD.tv.X, SD.tv.d, i, R, seed, SD.set, SD.hit, SD.l, SD.rowptr, SD.cV, SD.cA, SD.V, SD.col, SD.A, S, \
                  lane);                                                                                        \
    break;
    VD_FILL(1)
    VD_FILL(2)
    VD_FILL(3)
    VD_FILL(4)
    VD_FILL(5)
    VD_FILL(6)
    default:
      fill_item<8>(SD.tv.X, SD.tv.d, i, R, seed, SD.set, SD.hit, SD.l, SD.rowptr, SD.cV, SD.cA, SD.V, SD.col, SD.A, S,
                   lane);
      break;
#undef VD_FILL
  }
}

// Adds to acc the contribution of ray k of cell i (hit id, length lk) to
// dLoss/dx: for a node hit the vector along w (the row entry's P), for a face
// hit the component on the face's axis (x_i's own term).
template <int D>
__device__ __forceinline__ void adj_contrib(const double* X, int d, int64_t i, int64_t k, int32_t id, double lk,
                                            double gVi, double gAij, double cV, double cA, uint64_t seed,
                                            uint32_t set, const double* U, int64_t R, double (&acc)[D]) {
  double u[D];
  ray_dir<D>(U, seed, set, i, k, R, d, u);
  const double ld1 = ipow_d(lk, d - 1), ld = ipow_d(lk, d);
  if (id >= 0) {
    double w[D], ww = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) w[c] = c < d ? __dadd_rn(X[(int64_t)id * d + c], -X[i * d + c]) : 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c)
      if (c < d) ww = __dadd_rn(ww, __dmul_rn(w[c], w[c]));
    const double inw = rsqrt(ww);
    // the saved length is l = |w|^2 / (2 u.w) (Eq. (t) with v = g), so
    // 1 / (u.w) = 2 l / |w|^2 up to one rounding of l
    const double iden = 2.0 * lk / ww;
    const double c1 = 2.0 * (double)d * ld1 * inw, c2 = 2.0 * ld * inw * inw * inw;
    const double kV = gVi * cV * (double)d * ld1, kA = gAij * cA;
#pragma unroll
    for (int c = 0; c < D; ++c)
      if (c < d) {
        const double dl = (w[c] - lk * u[c]) * iden;
        acc[c] += kV * dl + kA * (c1 * dl - c2 * w[c]);
      }
  } else {
    const int a = face_axis(id);
    double ua = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c)
      if (c == a) ua = u[c];
    const double dl = -1.0 / ua;
    const double dadl = (d >= 2) ? (double)(d - 1) * ipow_d(lk, d - 2) / fabs(ua) : 0.0;
    const double G = gVi * cV * (double)d * ld1 * dl + gAij * cA * dadl * dl;
#pragma unroll
    for (int c = 0; c < D; ++c)
      if (c == a) acc[c] += G;
  }
}

// Row pass for rows with more entries than the sorted path holds: the rays
// of each entry gathered in one pass over the row per entry (L: room for
// kAdjList ray indices).
template <int D>
__device__ void adj_rows_by_id(const double* X, int d, int64_t i, int64_t R, uint64_t seed, uint32_t set,
                               const int32_t* h, const double* li, int64_t q0, int64_t nnz, const int32_t* col,
                               double cV, double cA, double gVi, const double* gA, double* P, double* own,
                               const double* U, int32_t* L, int lane) {
  double faceacc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) faceacc[c] = 0.0;
  for (int64_t q = q0; q < q0 + nnz; ++q) {
    const int32_t id = col[q];
    const double gAij = gA ? gA[q] : 0.0;
    double acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0.0;
    if (id >= 0) {
      // node hit: every ray adds a_k w - b_k u_k (w = x_j - x_i is the entry's),
      // so the rays accumulate the scalar sum of a_k and the vector of b_k u_k
      double w[D], ww = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) w[c] = c < d ? __dadd_rn(X[(int64_t)id * d + c], -X[i * d + c]) : 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (c < d) ww = __dadd_rn(ww, __dmul_rn(w[c], w[c]));
      const double inw = rsqrt(ww);
      const double kA = gAij * cA;
      const double cwa = 2.0 * (double)d * inw, cwb = 2.0 * inw * inw * inw;
      // 1 / (u.w) = 2 l / |w|^2 for every ray of the entry (l = |w|^2 / (2 u.w))
      const double c2w = 2.0 / ww;
      const double cg = gVi * cV * (double)d + kA * cwa;
      double asum = 0.0, bu[D];
#pragma unroll
      for (int c = 0; c < D; ++c) bu[c] = 0.0;
      int64_t k0 = 0;
      while (k0 < R) {
        const int m = gather_rays<kAdjList>(h, R, id, &k0, L, lane);
        for (int p = lane; p < m; p += 32) {
          const int32_t k = L[p];
          const double lk = li[k];
          double u[D];
          ray_dir<D>(U, seed, set, i, k, R, d, u);
          const double ld1 = ipow_d(lk, d - 1), ld = ld1 * lk;
          const double g = cg * ld * c2w;  // coefficient of dl: (gV cV d + kA cwa) l^(d-1) / (u.w)
          asum += g - kA * cwb * ld;
          const double b = g * lk;
#pragma unroll
          for (int c = 0; c < D; ++c) bu[c] += b * u[c];
        }
        __syncwarp();
      }
      asum = warp_sum_d(asum);
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] = c < d ? asum * w[c] - warp_sum_d(bu[c]) : 0.0;
    } else {
      int64_t k0 = 0;
      while (k0 < R) {
        const int m = gather_rays<kAdjList>(h, R, id, &k0, L, lane);
        for (int p = lane; p < m; p += 32) {
          const int32_t k = L[p];
          adj_contrib<D>(X, d, i, k, id, li[k], gVi, gAij, cV, cA, seed, set, U, R, acc);
        }
        __syncwarp();
      }
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] = warp_sum_d(acc[c]);
    }
    if (id >= 0) {
      if (lane == 0)
        for (int c = 0; c < d; ++c) P[q * d + c] = acc[c];
#pragma unroll
      for (int c = 0; c < D; ++c) faceacc[c] -= acc[c];
    } else {
      if (lane == 0)
        for (int c = 0; c < d; ++c) P[q * d + c] = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) faceacc[c] += acc[c];
    }
  }
  if (lane == 0)
    for (int c = 0; c < d; ++c) own[i * d + c] = faceacc[c];
}

// Row pass of the adjoint: P[q][*] = sum over the rays of cell i that hit
// col[q] of dLoss/dw (node) ; own[i][*] = face terms of x_i minus the node
// entries.  Rows with many rays per entry are sorted by entry: every lane
// sums a range of the sorted node rays (the scalar a_k and the vector
// b_k u_k of each entry, P = (sum a_k) w - sum b_k u_k), face entries take a
// warp each.  Rows with few rays per entry compute 32 rays at once and add
// them per entry in ascending ray order, the lanes splitting the components.
template <int D>
__global__ void __launch_bounds__(kMcWarps * 32) k_mc_adj_rows(const double* X, int64_t N, int d, int64_t R,
                                                               uint64_t seed, uint32_t set, const int32_t* hit,
                                                               const double* l, const int64_t* rowptr,
                                                               const int32_t* col, double cV, double cA,
                                                               const double* gV, const double* gA, double* P,
                                                               double* own, const double* U) {
  extern __shared__ __align__(16) unsigned char row_smem[];
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  using Scratch = RowScratch<D + 1, kAdjList>;
  Scratch& S = reinterpret_cast<Scratch*>(row_smem)[threadIdx.x >> 5];
  // per-entry factors of the sorted path, after the block's scratch array
  double(*cst)[2] = reinterpret_cast<double(*)[2]>(row_smem + kMcWarps * sizeof(Scratch)) + (threadIdx.x >> 5) * kEnt;
  const int32_t* h = hit + i * R;
  const double* li = l + i * R;
  const double gVi = gV[i];
  const int64_t q0 = rowptr[i], nnz = rowptr[i + 1] - q0;
  if (nnz * kFewRays > R) {
    double(*Cs)[D + 1] = S.acc;
    int32_t* Es = S.Ej;
    for (int64_t e = lane; e < nnz * d; e += 32) P[q0 * d + e] = 0.0;
    __syncwarp();
    for (int64_t k0 = 0; k0 < R; k0 += 32) {
      const int64_t k = k0 + lane;
      if (k < R) {
        const int32_t id = h[k];
        const int64_t q = entry_of(col, q0, nnz, id);
        double v[D];
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = 0.0;
        adj_contrib<D>(X, d, i, k, id, li[k], gVi, gA ? gA[q] : 0.0, cV, cA, seed, set, U, R, v);
#pragma unroll
        for (int c = 0; c < D; ++c) Cs[lane][c] = v[c];
        Es[lane] = (int32_t)(q - q0);
      }
      __syncwarp();
      if (lane < d)
        for (int r = 0; r < 32 && k0 + r < R; ++r) {
          double* pe = P + (q0 + Es[r]) * d + lane;
          *pe += Cs[r][lane];
        }
      __syncwarp();
    }
    if (lane < d) {  // x_i's own term: minus its node entries, plus its face entries, in entry order
      double o = 0.0;
      for (int64_t e = 0; e < nnz; ++e) {
        const double v = P[(q0 + e) * d + lane];
        o = col[q0 + e] >= 0 ? o - v : o + v;
      }
      own[i * d + lane] = o;
    }
    __syncwarp();
    for (int64_t e = lane; e < nnz; e += 32)
      if (col[q0 + e] < 0)
        for (int c = 0; c < d; ++c) P[(q0 + e) * d + c] = 0.0;
    return;
  }
  if (nnz > kEnt) {  // more entries than the sorted path holds: one pass over the row per entry
    adj_rows_by_id<D>(X, d, i, R, seed, set, h, li, q0, nnz, col, cV, cA, gVi, gA, P, own, U, S.Ej, lane);
    return;
  }
  // per-entry factors: node entries a_k = c0 l^d - c1 l^d, b_k = c0 l^(d+1)
  // (from 1 / (u.w) = 2 l / |w|^2), face entries keep gA
  for (int e = lane; e < nnz; e += 32) {
    const int32_t id = col[q0 + e];
    S.col[e] = id;
    const double gAij = gA ? gA[q0 + e] : 0.0;
    if (id >= 0) {
      double ww = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (c < d) {
          const double w = __dadd_rn(X[(int64_t)id * d + c], -X[i * d + c]);
          ww = __dadd_rn(ww, __dmul_rn(w, w));
        }
      const double inw = rsqrt(ww);
      const double kA = gAij * cA;
      const double cwa = 2.0 * (double)d * inw, cwb = 2.0 * inw * inw * inw;
      const double cg = gVi * cV * (double)d + kA * cwa;
      cst[e][0] = cg * (2.0 / ww);
      cst[e][1] = kA * cwb;
    } else {
      cst[e][0] = gAij;
      cst[e][1] = 0.0;
    }
  }
  __syncwarp();
  int nfe = 0;  // face entries (negative ids) come first
  for (int e0 = 0; e0 < nnz; e0 += 32) nfe += __popc(__ballot_sync(kFull, e0 + lane < nnz && S.col[e0 + lane] < 0));
  for (int64_t k0 = 0; k0 < R; k0 += kAdjList) {
    const int C = R - k0 < kAdjList ? (int)(R - k0) : kAdjList;
    const bool fst = k0 == 0;
    sort_chunk<D + 1>(h, k0, C, (int)nnz, S, lane);
    if (fst)
      for (int e = lane; e < nnz; e += 32)
#pragma unroll
        for (int v = 0; v <= D; ++v) S.acc[e][v] = 0.0;
    __syncwarp();
    for (int e = 0; e < nfe; ++e) {  // face entries: the term on the face's axis, a warp per entry
      const int s0 = S.st[e], n = S.cnt[e];
      if (n == 0) continue;
      const int32_t id = S.col[e];
      const int a = face_axis(id);
      double r[1] = {0.0};
      for (int p = s0 + lane; p < s0 + n; p += 32) {
        const int64_t k = k0 + S.L[p];
        double v[D];
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = 0.0;
        adj_contrib<D>(X, d, i, k, id, li[k], gVi, cst[e][0], cV, cA, seed, set, U, R, v);
#pragma unroll
        for (int c = 0; c < D; ++c)
          if (c == a) r[0] = __dadd_rn(r[0], v[c]);
      }
      r[0] = warp_sum_d(r[0]);
      if (lane == 0) put_acc<D + 1, 1>(S.acc[e], r, fst);
    }
    __syncwarp();
    const int F0 = nfe < nnz ? S.st[nfe] : C;
    seg_sums<D + 1, D + 1>(S, F0, C, fst, lane, [&](double (&run)[D + 1], bool reset, int e, int j) {
      const int64_t k = k0 + j;
      const double lk = li[k];
      double u[D];
      ray_dir<D>(U, seed, set, i, k, R, d, u);
      const double ld = __dmul_rn(ipow_d(lk, d - 1), lk);
      const double g = __dmul_rn(cst[e][0], ld);
      const double b = __dmul_rn(g, lk);
      run[0] = __dadd_rn(reset ? 0.0 : run[0], __fma_rn(-cst[e][1], ld, g));
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (c < d) run[1 + c] = __fma_rn(b, u[c], reset ? 0.0 : run[1 + c]);
    });
  }
  // P of the node entries; every entry's vector for x_i's own term
  for (int e = lane; e < nnz; e += 32) {
    const int64_t q = q0 + e;
    const int32_t id = S.col[e];
    if (id >= 0) {
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (c < d) {
          const double w = __dadd_rn(X[(int64_t)id * d + c], -X[i * d + c]);
          const double v = __fma_rn(S.acc[e][0], w, -S.acc[e][1 + c]);
          P[q * d + c] = v;
          S.acc[e][1 + c] = v;
        }
    } else {
      const int a = face_axis(id);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (c < d) P[q * d + c] = 0.0;
        S.acc[e][1 + c] = c == a ? S.acc[e][0] : 0.0;
      }
    }
  }
  __syncwarp();
  if (lane < d) {  // minus the node entries, plus the face entries, in entry order
    double o = 0.0;
    for (int e = 0; e < nnz; ++e) {
      const double v = S.acc[e][1 + lane];
      o = S.col[e] >= 0 ? __dadd_rn(o, -v) : __dadd_rn(o, v);
    }
    own[i * d + lane] = o;
  }
}

// keys: column (node id) of each node entry, vals: entry index
__global__ void k_mc_col_keys(const int32_t* col, int64_t nnz, uint64_t* keys, int32_t* vals) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nnz) return;
  const int32_t c = col[q];
  keys[q] = c >= 0 ? (uint64_t)c : (uint64_t)0xFFFFFFFFull;  // faces sort last
  vals[q] = (int32_t)q;
}

// column pass: gX[j] = own[j] + sum over entries (i, j) in ascending i of P
__global__ void k_mc_adj_cols(const uint64_t* keys, const int32_t* vals, int64_t nnz, const double* P,
                              const double* own, int64_t N, int d, double* gX) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  // binary search the first entry with key j
  int64_t lo = 0, hi = nnz;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (keys[mid] < (uint64_t)j) lo = mid + 1;
    else hi = mid;
  }
  double acc[VD_MAX_D];
  for (int c = 0; c < d; ++c) acc[c] = own[j * d + c];
  for (int64_t q = lo; q < nnz && keys[q] == (uint64_t)j; ++q) {
    const int64_t e = vals[q];
    for (int c = 0; c < d; ++c) acc[c] += P[e * d + c];
  }
  for (int c = 0; c < d; ++c) gX[j * d + c] = acc[c];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

template <int D>
cudaError_t fill_d(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set, const int32_t* hit,
                   const double* l, const int64_t* rowptr, double cV, double cA, double* V, int32_t* col, double* A,
                   const double* U, cudaStream_t st) {
  const size_t sm = kMcWarps * sizeof(RowScratch<2>);
  cudaError_t e = cudaFuncSetAttribute(k_mc_fill<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_mc_fill<D><<<nblk(N * 32, kMcWarps * 32), kMcWarps * 32, sm, st>>>(X, N, d, R, seed, set, hit, l, rowptr, cV, cA,
                                                                       V, col, A, U);
  count_launch();
  return cudaGetLastError();
}

template <int D>
cudaError_t adj_rows_d(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set,
                       const int32_t* hit, const double* l, const int64_t* rowptr, const int32_t* col, double cV,
                       double cA, const double* gV, const double* gA, double* P, double* own, const double* U,
                       cudaStream_t st) {
  const size_t sm = kMcWarps * (sizeof(RowScratch<D + 1, kAdjList>) + kEnt * 2 * sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(k_mc_adj_rows<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_mc_adj_rows<D><<<nblk(N * 32, kMcWarps * 32), kMcWarps * 32, sm, st>>>(X, N, d, R, seed, set, hit, l, rowptr,
                                                                           col, cV, cA, gV, gA, P, own, U);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

double sphere_area(int d) { return 2.0 * std::pow(M_PI, 0.5 * d) / std::tgamma(0.5 * d); }

cudaError_t mc_batch_reduce(const SetDesc* sets_dev, int nsets, int64_t nitems, int maxd, int64_t R, uint64_t seed,
                            cudaStream_t st) {
  (void)maxd;
  k_mc_count_batch<<<nblk(nitems * 32, 128), 128, 0, st>>>(sets_dev, nsets, nitems, R);
  count_launch();
  k_scan_batch<<<nsets, 1024, 0, st>>>(sets_dev);
  count_launch();
  const size_t sm = kMcWarps * sizeof(RowScratch<2>);
  cudaError_t e = cudaFuncSetAttribute(k_mc_fill_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_mc_fill_batch<<<nblk(nitems * 32, kMcWarps * 32), kMcWarps * 32, sm, st>>>(sets_dev, nsets, nitems, R, seed);
  count_launch();
  return cudaGetLastError();
}

// out[0..n] = exclusive scan of in[0..n) (out[n] = total), one block.
cudaError_t mc_scan64(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st) {
  k_scan64<<<1, 1024, 0, st>>>(in, n, out);
  count_launch();
  return cudaGetLastError();
}

// Counts the distinct hits per cell and writes rowptr (N+1); returns nnz.
cudaError_t mc_rowptr(const int32_t* hit, int64_t N, int64_t R, int64_t* cnt_scratch, int64_t* rowptr,
                      int64_t* nnz_host, cudaStream_t st) {
  k_mc_count<<<nblk(N * 32, 128), 128, 0, st>>>(hit, N, R, cnt_scratch); count_launch();
  k_scan64<<<1, 1024, 0, st>>>(cnt_scratch, N, rowptr); count_launch();
  cudaMemcpyAsync(nnz_host, rowptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t mc_fill(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set, const int32_t* hit,
                    const double* l, const int64_t* rowptr, double* V, int32_t* col, double* A, const double* U,
                    cudaStream_t st) {
  const double S = sphere_area(d);
  const double cV = S / ((double)d * (double)R), cA = S / (double)R;
  if (d <= 4) return fill_d<4>(X, N, d, R, seed, set, hit, l, rowptr, cV, cA, V, col, A, U, st);
  if (d <= 8) return fill_d<8>(X, N, d, R, seed, set, hit, l, rowptr, cV, cA, V, col, A, U, st);
  return fill_d<16>(X, N, d, R, seed, set, hit, l, rowptr, cV, cA, V, col, A, U, st);
}

cudaError_t mc_integrals(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set,
                         const int32_t* hit, const double* l, const int64_t* rowptr, const int32_t* col,
                         const double* U, const vd_func& f, int64_t m, double* FV, double* Fd, cudaStream_t st) {
  const double S = sphere_area(d);
  const double cV = S / ((double)R * (double)m), cA = S / (double)R;
  const unsigned g = nblk(N * 32, kMcWarps * 32);
  const size_t sm = kMcWarps * sizeof(RowScratch<1>);
  cudaError_t e = cudaSuccess;
  if (d <= 4) {
    if ((e = cudaFuncSetAttribute(k_mc_func<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) == cudaSuccess)
      k_mc_func<4><<<g, kMcWarps * 32, sm, st>>>(X, N, d, R, seed, set, hit, l, rowptr, col, U, f, m, cV, cA, FV, Fd);
  } else if (d <= 8) {
    if ((e = cudaFuncSetAttribute(k_mc_func<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) == cudaSuccess)
      k_mc_func<8><<<g, kMcWarps * 32, sm, st>>>(X, N, d, R, seed, set, hit, l, rowptr, col, U, f, m, cV, cA, FV, Fd);
  } else {
    if ((e = cudaFuncSetAttribute(k_mc_func<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) == cudaSuccess)
      k_mc_func<16><<<g, kMcWarps * 32, sm, st>>>(X, N, d, R, seed, set, hit, l, rowptr, col, U, f, m, cV, cA, FV, Fd);
  }
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaGetLastError();
}

cudaError_t mc_adjoint(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set,
                       const int32_t* hit, const double* l, const int64_t* rowptr, const int32_t* col, int64_t nnz,
                       const double* gV, const double* gA, double* gX, const double* U, DevBufs& scratch,
                       cudaStream_t st) {
  const double S = sphere_area(d);
  const double cV = S / ((double)d * (double)R), cA = S / (double)R;
  double *P = nullptr, *own = nullptr;
  uint64_t *keys = nullptr, *ktmp = nullptr;
  int32_t *vals = nullptr, *vtmp = nullptr;
  uint32_t* counts = nullptr;
  unsigned long long* orand = nullptr;
  cudaError_t e;
  const int64_t nn = std::max<int64_t>(nnz, 1);
  if ((e = scratch.alloc_n(&P, (size_t)nn * d)) != cudaSuccess || (e = scratch.alloc_n(&own, (size_t)N * d)) ||
      (e = scratch.alloc_n(&keys, nn)) || (e = scratch.alloc_n(&ktmp, nn)) || (e = scratch.alloc_n(&vals, nn)) ||
      (e = scratch.alloc_n(&vtmp, nn)) || (e = scratch.alloc_n(&counts, (size_t)256 * (nn / 4096 + 2))) ||
      (e = scratch.alloc_n(&orand, 2)))
    return e;
  if (d <= 4) e = adj_rows_d<4>(X, N, d, R, seed, set, hit, l, rowptr, col, cV, cA, gV, gA, P, own, U, st);
  else if (d <= 8) e = adj_rows_d<8>(X, N, d, R, seed, set, hit, l, rowptr, col, cV, cA, gV, gA, P, own, U, st);
  else e = adj_rows_d<16>(X, N, d, R, seed, set, hit, l, rowptr, col, cV, cA, gV, gA, P, own, U, st);
  if (e != cudaSuccess) return e;
  k_mc_col_keys<<<nblk(nnz, 256), 256, 0, st>>>(col, nnz, keys, vals); count_launch();
  e = radix_sort_u64(keys, vals, ktmp, vtmp, nnz, counts, orand, st);
  if (e != cudaSuccess) return e;
  k_mc_adj_cols<<<nblk(N, 128), 128, 0, st>>>(keys, vals, nnz, P, own, N, d, gX); count_launch();
  return cudaGetLastError();
}

}  // namespace vd
