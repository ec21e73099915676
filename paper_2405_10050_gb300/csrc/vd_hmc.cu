// vd_hmc.cu -- heuristic Monte Carlo integration (Section 3.3) on the GPU:
// from the interface areas A_ij of an MC run and the vertices of the diagram
// (the traversal's sorted tuples and coordinates),
//   V_i  = (1/d) sum_j h_ij A_ij,
//   F_ij = (d/(d+1)) (1/K_ij) sum_k f(nu_k) A_ij + (1/(d+1)) f(y_ij) A_ij,
//   I_i  = sum_j (h_ij/d) ((d/(d+1)) F_ij + (1/(d+1)) A_ij f(x_i)),
// with nu_k the K_ij vertices whose tuple holds both i and j, y_ij their
// mean, h_ij = |x_j - x_i|/2 or the distance from x_i to the box face j; the
// last line is the cone rule of Eq. (leibniz-int) over the pyramid with base
// facet ij and apex x_i.
//
// Work layout: every (vertex, ordered pair (i, j) of its tuple, i a node)
// whose (i, j) is an entry of the CSR is one contribution.  A counting pass
// sizes each entry's list, a fill pass writes the vertex ids (in any order),
// then one thread per entry sorts its list (ascending vertex id) and sums
// over it in that order, and one thread per cell sums over its row: every
// sum has a fixed order, the one of the oracle.
#include <algorithm>
#include <cmath>

#include "vd_dev.cuh"

namespace vd {

namespace {

// position of id in row i of the CSR (col ascending), -1 if absent
__device__ __forceinline__ int64_t row_find(const int64_t* rowptr, const int32_t* col, int64_t i, int32_t id) {
  int64_t lo = rowptr[i], hi = rowptr[i + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (col[mid] < id) lo = mid + 1;
    else hi = mid;
  }
  return (lo < rowptr[i + 1] && col[lo] == id) ? lo : -1;
}

// f at y, binary64 in the operation order of include/vd.h
__device__ double hmc_f(const vd_func& f, int d, const double* y) {
  if (f.kind == VD_F_POLY2) {
    double s = f.c0;
    for (int a = 0; a < d; ++a) s = __dadd_rn(s, __dmul_rn(f.b[a], y[a]));
    for (int a = 0; a < d; ++a) s = __dadd_rn(s, __dmul_rn(f.q[a], __dmul_rn(y[a], y[a])));
    return s;
  }
  if (f.kind == VD_F_SIN_SQ) return sin(__dmul_rn(y[f.axis], y[f.axis]));
  return 1.0;
}

// mode 0: count the contributions of each entry (cnt); mode 1: write vertex
// ids into the entries' lists (off = list starts, cnt = cursors from 0)
__global__ void k_hmc_pairs(const int32_t* tuples, int64_t nv, int d, int64_t N, const int64_t* rowptr,
                            const int32_t* col, unsigned long long* cnt, const int64_t* off, int32_t* vids,
                            int mode) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int32_t* sg = tuples + v * (d + 1);
  for (int a = 0; a <= d; ++a) {
    const int32_t i = sg[a];
    if (i < 0 || i >= N) continue;
    for (int b = 0; b <= d; ++b) {
      if (b == a) continue;
      const int64_t e = row_find(rowptr, col, i, sg[b]);
      if (e < 0) continue;
      const unsigned long long k = atomicAdd(&cnt[e], 1ull);
      if (mode == 1) vids[off[e] + (int64_t)k] = (int32_t)v;
    }
  }
}

// one thread per entry: sort its vertex list, then K, sum f, mean y, F_ij
__global__ void k_hmc_entries(const double* coords, int d, const int64_t* off, int32_t* vids, const double* A,
                              int64_t nnz, vd_func f, double cd, double c1, double* FH) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int64_t lo = off[e], hi = off[e + 1];
  for (int64_t p = lo + 1; p < hi; ++p) {  // insertion sort: the lists are short
    const int32_t x = vids[p];
    int64_t q = p - 1;
    while (q >= lo && vids[q] > x) {
      vids[q + 1] = vids[q];
      --q;
    }
    vids[q + 1] = x;
  }
  double F = 0.0;
  if (hi > lo) {
    double fs = 0.0, ys[VD_MAX_D];
    for (int c = 0; c < d; ++c) ys[c] = 0.0;
    for (int64_t p = lo; p < hi; ++p) {
      const double* nu = coords + (int64_t)vids[p] * d;
      fs = __dadd_rn(fs, hmc_f(f, d, nu));
      for (int c = 0; c < d; ++c) ys[c] = __dadd_rn(ys[c], nu[c]);
    }
    const double K = (double)(hi - lo);
    for (int c = 0; c < d; ++c) ys[c] = __ddiv_rn(ys[c], K);
    const double mf = __ddiv_rn(fs, K);
    F = __dmul_rn(__dadd_rn(__dmul_rn(cd, mf), __dmul_rn(c1, hmc_f(f, d, ys))), A[e]);
  }
  FH[e] = F;
}

// one thread per cell: V_i and I_i over its row in CSR order
__global__ void k_hmc_cells(const double* X, int64_t N, int d, const int64_t* rowptr, const int32_t* col,
                            const double* A, const double* FH, vd_func f, double cd, double c1, double* VH,
                            double* IH) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* xi = X + i * d;
  const double fxi = hmc_f(f, d, xi);
  const double dd = (double)d;
  double vh = 0.0, ih = 0.0;
  for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int32_t j = col[e];
    double h;
    if (j >= 0) {
      double ww = 0.0;
      for (int c = 0; c < d; ++c) {
        const double w = __dadd_rn(X[(int64_t)j * d + c], -xi[c]);
        ww = __dadd_rn(ww, __dmul_rn(w, w));
      }
      h = __dmul_rn(0.5, __dsqrt_rn(ww));
    } else {
      const double xa = xi[face_axis(j)];
      h = face_side(j) ? __dadd_rn(1.0, -xa) : xa;
    }
    vh = __dadd_rn(vh, __dmul_rn(h, A[e]));
    ih = __dadd_rn(ih, __dmul_rn(__ddiv_rn(h, dd), __dadd_rn(__dmul_rn(cd, FH[e]), __dmul_rn(c1, __dmul_rn(A[e], fxi)))));
  }
  if (VH) VH[i] = __ddiv_rn(vh, dd);
  if (IH) IH[i] = ih;
}

__global__ void k_u64_to_i64(const unsigned long long* in, int64_t n, int64_t* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int64_t)in[i];
}

inline unsigned nb(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t mc_scan64(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st);

// FH must hold nnz values (scratch if the caller wants none).
cudaError_t hmc_integrals(const double* X, int64_t N, int d, const int64_t* rowptr, const int32_t* col,
                          const double* A, int64_t nnz, const int32_t* tuples, const double* coords, int64_t nv,
                          const vd_func& f, double* VH, double* FH, double* IH, DevBufs& scratch, cudaStream_t st) {
  const double cd = (double)d / (double)(d + 1), c1 = 1.0 / (double)(d + 1);
  const int64_t nn = std::max<int64_t>(nnz, 1);
  unsigned long long* cnt = nullptr;
  int64_t *cnt64 = nullptr, *off = nullptr;
  int32_t* vids = nullptr;
  cudaError_t e;
  if ((e = scratch.alloc_n(&cnt, (size_t)nn)) || (e = scratch.alloc_n(&cnt64, (size_t)nn)) ||
      (e = scratch.alloc_n(&off, (size_t)nn + 1)))
    return e;
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * nn, st))) return e;
  if (nv > 0) {
    k_hmc_pairs<<<nb(nv, 128), 128, 0, st>>>(tuples, nv, d, N, rowptr, col, cnt, nullptr, nullptr, 0);
    count_launch();
  }
  k_u64_to_i64<<<nb(nnz, 256), 256, 0, st>>>(cnt, nnz, cnt64);
  count_launch();
  if ((e = mc_scan64(cnt64, nnz, off, st))) return e;
  int64_t total = 0;
  if ((e = cudaMemcpyAsync(&total, off + nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  if ((e = scratch.alloc_n(&vids, (size_t)std::max<int64_t>(total, 1)))) return e;
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * nn, st))) return e;
  if (nv > 0) {
    k_hmc_pairs<<<nb(nv, 128), 128, 0, st>>>(tuples, nv, d, N, rowptr, col, cnt, off, vids, 1);
    count_launch();
  }
  k_hmc_entries<<<nb(nnz, 128), 128, 0, st>>>(coords, d, off, vids, A, nnz, f, cd, c1, FH);
  count_launch();
  k_hmc_cells<<<nb(N, 128), 128, 0, st>>>(X, N, d, rowptr, col, A, FH, f, cd, c1, VH, IH);
  count_launch();
  return cudaGetLastError();
}

}  // namespace vd
