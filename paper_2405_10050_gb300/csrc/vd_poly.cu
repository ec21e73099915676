// vd_poly.cu -- exact cell volumes, interface areas and integrals of the
// piecewise linear interpolant of f from the vertices of the diagram
// (Section 3.2, Algorithms 4-5, IterativeVolume).
//
// For cell i the faces are walked depth first, one thread per facet: level 1
// is the cell (the vertices whose tuple holds i, ascending), the face at
// level D+1 keeps the vertices of its parent whose tuple holds the generator
// j that defines it (candidates in ascending id, not yet in the face), down
// to the edges at level d, which have exactly two vertices nu < nu'.  Every
// edge closes the simplex (x_i, m_2, ..., m_{d-1}, nu, nu'), m_D the mean of
// the level-D face's vertices, of volume |det(m_2 - x_i, ..., nu - x_i,
// nu' - x_i)| / d! (Gaussian elimination, partial pivoting on the first
// maximal |entry|).  Integrals take Algorithm 5's weights: an edge returns
// F = (f(nu) + f(nu'))/2 V, a face at level D the sum of its children's V
// and ((d-D+1)/(d-D+2)) sum F + (1/(d-D+2)) f(m_D) sum V, the cell
// F_i = (d/(d+1)) sum F + (1/(d+1)) f(x_i) sum V; a facet ij gives
// A_ij = V_ij d / h_ij and Fd_ij = F_ij d / h_ij.  Binary64 with the
// operations in that order, so polynomial f reproduces the oracle bit for
// bit.  One thread walks the pyramid over one facet (levels 2..d, its vertex
// lists in scratch of (d-1) times the facet's vertex count); a thread per
// cell then sums its pyramids in facet order.
#include <algorithm>
#include <cmath>

#include "vd_dev.cuh"

namespace vd {

cudaError_t radix_sort_u64(uint64_t* keys, int32_t* vals, uint64_t* ktmp, int32_t* vtmp, int64_t n,
                           uint32_t* counts, unsigned long long* orand, cudaStream_t st);
cudaError_t mc_scan64(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st);

namespace {

constexpr int kLzMaxD = 8;
constexpr unsigned kLzFlagDegenerate = 1u;

__device__ double lz_f(const vd_func& f, int d, const double* y) {
  if (f.kind == VD_F_POLY2) {
    double s = f.c0;
    for (int a = 0; a < d; ++a) s = __dadd_rn(s, __dmul_rn(f.b[a], y[a]));
    for (int a = 0; a < d; ++a) s = __dadd_rn(s, __dmul_rn(f.q[a], __dmul_rn(y[a], y[a])));
    return s;
  }
  if (f.kind == VD_F_SIN_SQ) return sin(__dmul_rn(y[f.axis], y[f.axis]));
  return 1.0;
}

// smallest generator > prev in the tuples of list[0..n) outside S[0..ns),
// INT32_MAX if none: the warp's lanes scan interleaved entries, then a min
__device__ int32_t lz_next(const int32_t* tuples, int L, const int32_t* list, int n, const int32_t* S, int ns,
                           int64_t prev, int lane) {
  int32_t best = INT32_MAX;
  for (int q = lane; q < n; q += 32) {
    const int32_t* t = tuples + (int64_t)list[q] * L;
    for (int k = 0; k < L; ++k) {
      const int32_t g = t[k];
      if ((int64_t)g <= prev || g >= best) continue;
      bool in = false;
      for (int s = 0; s < ns; ++s) in |= (S[s] == g);
      if (!in) best = g;
    }
  }
  return __reduce_min_sync(kFull, best);
}

__device__ __forceinline__ bool lz_has(const int32_t* t, int L, int32_t g) {
  bool in = false;
  for (int k = 0; k < L; ++k) in |= (t[k] == g);
  return in;
}

// |det| of the d x d row-major matrix M (destroyed)
__device__ double lz_absdet(double* M, int d) {
  double det = 1.0;
  for (int c = 0; c < d; ++c) {
    int p = c;
    for (int r = c + 1; r < d; ++r)
      if (fabs(M[r * d + c]) > fabs(M[p * d + c])) p = r;
    if (M[p * d + c] == 0.0) return 0.0;
    if (p != c)
      for (int k = 0; k < d; ++k) {
        const double t = M[c * d + k];
        M[c * d + k] = M[p * d + k];
        M[p * d + k] = t;
      }
    for (int r = c + 1; r < d; ++r) {
      const double mlt = __ddiv_rn(M[r * d + c], M[c * d + c]);
      for (int k = c + 1; k < d; ++k) M[r * d + k] = __dadd_rn(M[r * d + k], -__dmul_rn(mlt, M[c * d + k]));
    }
    det = __dmul_rn(det, M[c * d + c]);
  }
  return fabs(det);
}

// keys[v (d+1) + k] = the cell of node tuples[v][k] (N for a box face), vals = v
__global__ void k_lz_pairs(const int32_t* tuples, int64_t nv, int d, int64_t N, uint64_t* keys, int32_t* vals,
                           unsigned long long* cnt) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nv * (d + 1)) return;
  const int32_t g = tuples[t];
  const bool node = g >= 0 && g < N;
  keys[t] = node ? (uint64_t)g : (uint64_t)N;
  vals[t] = (int32_t)(t / (d + 1));
  if (node) atomicAdd(&cnt[g], 1ull);
}

__global__ void k_lz_u64_to_i64(const unsigned long long* in, int64_t n, int64_t* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int64_t)in[i];
}

// A warp per cell.  mode 0: the number of facets of cell i (distinct
// generators other than i in its vertices' tuples); mode 1: their
// generators in ascending order into col (from rowptr[i]), the cell into
// erow and the facet's vertex count into m2.
__global__ void k_lz_facet_list(const int32_t* tuples, int d, int64_t N, const int64_t* voff, const int32_t* vlist,
                                int64_t* fcnt, const int64_t* rowptr, int32_t* col, int32_t* erow, int64_t* m2,
                                int mode) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  const int L = d + 1;
  const int32_t* L1 = vlist + voff[i];
  const int n1 = (int)(voff[i + 1] - voff[i]);
  const int32_t S0 = (int32_t)i;
  int64_t c = 0, j = INT64_MIN;
  int32_t jn;
  while ((jn = lz_next(tuples, L, L1, n1, &S0, 1, j, lane)) != INT32_MAX) {
    if (mode == 1) {
      int m = 0;
      for (int p = lane; p < n1; p += 32) m += lz_has(tuples + (int64_t)L1[p] * L, L, jn) ? 1 : 0;
      for (int o = 16; o; o >>= 1) m += __shfl_xor_sync(kFull, m, o);
      if (lane == 0) {
        const int64_t e = rowptr[i] + c;
        col[e] = jn;
        erow[e] = (int32_t)i;
        m2[e] = m;
      }
    }
    ++c;
    j = jn;
  }
  if (mode == 0 && lane == 0) fcnt[i] = c;
}

// Sort keys of the facets by decreasing vertex count (the stable sort keeps
// the CSR order among equal counts): a warp then walks pyramids of similar
// size.
__global__ void k_lz_order_keys(const int64_t* m2off, int64_t nnz, uint64_t* keys, int32_t* vals) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int64_t n2 = m2off[e + 1] - m2off[e];
  keys[e] = 0xFFFFFFFFull - (uint64_t)(n2 < 0xFFFFFFFFll ? n2 : 0xFFFFFFFFll);
  vals[e] = (int32_t)e;
}

// A warp per cell: the vertices of each facet (i, j) (the cell's vertices
// whose tuple holds j), in the cell's vertex order, at
// scratch + (d - 1) m2off[e]; the warp reads the cell's list once per facet.
__global__ void k_lz_facet_verts(const int32_t* tuples, int d, int64_t N, const int64_t* voff, const int32_t* vlist,
                                 const int64_t* rowptr, const int32_t* col, const int64_t* m2off, int32_t* scratch) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  const int L = d + 1;
  const int32_t* L1 = vlist + voff[i];
  const int n1 = (int)(voff[i + 1] - voff[i]);
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int32_t j = col[e];
    const int64_t n2 = m2off[e + 1] - m2off[e];
    int32_t* base = scratch + (int64_t)(d - 1) * m2off[e];
    int64_t m = 0;
    for (int p0 = 0; p0 < n1; p0 += 32) {
      const int p = p0 + lane;
      const bool has = p < n1 && lz_has(tuples + (int64_t)L1[p] * L, L, j);
      const unsigned b = __ballot_sync(kFull, has);
      const int64_t q = m + __popc(b & lt);
      if (has && q < n2) base[q] = L1[p];
      m += __popc(b);
    }
  }
}

// Facet (i, j), facet e = order[t] of position t (e = t without an order):
// the pyramid over it with apex x_i, walked from the facet (level 2) down to
// its edges; writes the pyramid's volume and integral (Vp, Fp) and the
// facet's A_ij, Fd_ij.
__device__ __forceinline__ void lz_facet(int64_t t, const double* X, int64_t N, int d, const int32_t* tuples,
                                         const double* coords, const int32_t* col, const int32_t* erow,
                                         const int64_t* m2off, const int32_t* order, int32_t* scratch, vd_func f,
                                         double fact, double* Vp, double* Fp, double* A, double* Fd,
                                         unsigned* flags) {
  const int64_t e = order ? order[t] : t;
  const int L = d + 1;
  const int64_t i = erow[e];
  const int32_t jf = col[e];
  const double* xi = X + i * d;
  const double dd = (double)d;
  const int n2 = (int)(m2off[e + 1] - m2off[e]);
  int32_t* base = scratch + (int64_t)(d - 1) * m2off[e];
  const int32_t* lst[kLzMaxD + 1];
  int cnt[kLzMaxD + 1];
  int64_t prev[kLzMaxD + 1];
  double sv[kLzMaxD + 1], sf[kLzMaxD + 1], fm[kLzMaxD + 1];
  double mid[kLzMaxD + 1][kLzMaxD];
  int32_t S[kLzMaxD + 1];
  double M[kLzMaxD * kLzMaxD];
  S[0] = (int32_t)i;
  S[1] = jf;
  const int m = n2;  // the facet's vertices, listed at base by k_lz_facet_verts
  // an edge closing a simplex with the current means: its (v, fv)
  auto edge = [&](const int32_t* child, int mm, double& v, double& fv) {
    v = fv = 0.0;
    if (mm != 2) {
      atomicOr(flags, kLzFlagDegenerate);
      return;
    }
    for (int c = 0; c < d; ++c) {
      const double* p = c < d - 2 ? mid[c + 2] : coords + (int64_t)child[c - (d - 2)] * d;
      for (int r = 0; r < d; ++r) M[r * d + c] = __dadd_rn(p[r], -xi[r]);
    }
    v = __ddiv_rn(lz_absdet(M, d), fact);
    const double f0 = lz_f(f, d, coords + (int64_t)child[0] * d), f1 = lz_f(f, d, coords + (int64_t)child[1] * d);
    fv = __dmul_rn(__dmul_rn(0.5, __dadd_rn(f0, f1)), v);
  };
  auto mean = [&](int D, const int32_t* lstD, int mm) {
    for (int a = 0; a < d; ++a) mid[D][a] = 0.0;
    for (int p = 0; p < mm; ++p)
      for (int a = 0; a < d; ++a) mid[D][a] = __dadd_rn(mid[D][a], coords[(int64_t)lstD[p] * d + a]);
    for (int a = 0; a < d; ++a) mid[D][a] = __ddiv_rn(mid[D][a], (double)mm);
    fm[D] = lz_f(f, d, mid[D]);
  };
  double Vpy = 0.0, Fpy = 0.0;
  if (d == 2) {  // the facet is an edge
    edge(base, m, Vpy, Fpy);
  } else {
    int D = 2;
    lst[2] = base;
    cnt[2] = m;
    prev[2] = INT64_MIN;
    sv[2] = sf[2] = 0.0;
    mean(2, base, m);
    while (true) {
      int32_t j = INT32_MAX;  // next candidate of level D
      for (int q = 0; q < cnt[D]; ++q) {
        const int32_t* t = tuples + (int64_t)lst[D][q] * L;
        for (int k = 0; k < L; ++k) {
          const int32_t g = t[k];
          if ((int64_t)g <= prev[D] || g >= j) continue;
          bool in = false;
          for (int s2 = 0; s2 < D; ++s2) in |= (S[s2] == g);
          if (!in) j = g;
        }
      }
      if (j == INT32_MAX) {  // level D is complete
        const double w1 = __ddiv_rn((double)(d - D + 1), (double)(d - D + 2)), w0 = __ddiv_rn(1.0, (double)(d - D + 2));
        const double fv = __dadd_rn(__dmul_rn(w1, sf[D]), __dmul_rn(__dmul_rn(w0, fm[D]), sv[D]));
        const double v = sv[D];
        if (D == 2) {
          Vpy = v;
          Fpy = fv;
          break;
        }
        --D;
        sv[D] = __dadd_rn(sv[D], v);
        sf[D] = __dadd_rn(sf[D], fv);
        continue;
      }
      prev[D] = j;
      S[D] = j;
      int32_t* child = base + (int64_t)(D - 1) * n2;
      int mm = 0;
      for (int p = 0; p < cnt[D]; ++p)
        if (lz_has(tuples + (int64_t)lst[D][p] * L, L, j)) child[mm++] = lst[D][p];
      if (D + 1 == d) {
        double v, fv;
        edge(child, mm, v, fv);
        sv[D] = __dadd_rn(sv[D], v);
        sf[D] = __dadd_rn(sf[D], fv);
        continue;
      }
      ++D;
      lst[D] = child;
      cnt[D] = mm;
      prev[D] = INT64_MIN;
      sv[D] = sf[D] = 0.0;
      mean(D, child, mm);
    }
  }
  double h = 1.0;
  if (jf >= N || (jf < 0 && face_axis(jf) >= d)) {  // not a generator of this node set
    atomicOr(flags, kLzFlagDegenerate);
  } else if (jf >= 0) {
    double ww = 0.0;
    for (int a = 0; a < d; ++a) {
      const double w = __dadd_rn(X[(int64_t)jf * d + a], -xi[a]);
      ww = __dadd_rn(ww, __dmul_rn(w, w));
    }
    h = __dmul_rn(0.5, __dsqrt_rn(ww));
  } else {
    const double xa = xi[face_axis(jf)];
    h = face_side(jf) ? __dadd_rn(1.0, -xa) : xa;
  }
  Vp[e] = Vpy;
  Fp[e] = Fpy;
  A[e] = __ddiv_rn(__dmul_rn(Vpy, dd), h);
  Fd[e] = __ddiv_rn(__dmul_rn(Fpy, dd), h);
}

// One thread per facet: each warp claims the next 32 positions until none is
// left, so the walk's long tail spreads over the SMs whatever the number of
// waves a one-shot grid would take.
__global__ void k_lz_facets(const double* X, int64_t N, int d, const int32_t* tuples, const double* coords,
                            const int32_t* col, const int32_t* erow, const int64_t* m2off, int64_t nnz,
                            const int32_t* order, int32_t* scratch, vd_func f, double fact, double* Vp, double* Fp,
                            double* A, double* Fd, unsigned* flags, unsigned long long* work) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long t0 = 0;
    if (lane == 0) t0 = atomicAdd(work, 32ull);
    t0 = __shfl_sync(kFull, t0, 0);
    if (t0 >= (unsigned long long)nnz) return;
    const int64_t t = (int64_t)t0 + lane;
    if (t < nnz) lz_facet(t, X, N, d, tuples, coords, col, erow, m2off, order, scratch, f, fact, Vp, Fp, A, Fd, flags);
    __syncwarp();
  }
}

// one thread per cell: V_i and F_i from its pyramids in facet order
__global__ void k_lz_cellsum(const double* X, int64_t N, int d, const int64_t* rowptr, const double* Vp,
                             const double* Fp, vd_func f, double* V, double* F) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double sv = 0.0, sf = 0.0;
  for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    sv = __dadd_rn(sv, Vp[e]);
    sf = __dadd_rn(sf, Fp[e]);
  }
  const double dd = (double)d;
  const double cd = __ddiv_rn(dd, (double)(d + 1)), c1 = __ddiv_rn(1.0, (double)(d + 1));
  V[i] = sv;
  F[i] = __dadd_rn(__dmul_rn(cd, sf), __dmul_rn(__dmul_rn(c1, lz_f(f, d, X + i * d)), sv));
}

inline unsigned nb(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

// Exact integration of the node set X (N x d, device) from the vertices
// (tuples, coords: nv rows, device).  Allocates the outputs from `out`
// (V, F: N; rowptr: N+1; col, A, Fd: *nnz) and its scratch from `scratch`.
cudaError_t poly_integrate(const double* X, int64_t N, int d, const int32_t* tuples, const double* coords,
                           int64_t nv, const vd_func& f, DevBufs& out, DevBufs& scratch, double** V, double** F,
                           int64_t** rowptr, int32_t** col, double** A, double** Fd, int64_t* nnz, unsigned* flags_h,
                           cudaStream_t st) {
  if (d < 2 || d > kLzMaxD) return cudaErrorInvalidValue;
  cudaError_t e;
  const int64_t np = std::max<int64_t>(nv * (d + 1), 1);
  uint64_t *keys = nullptr, *ktmp = nullptr;
  int32_t *vals = nullptr, *vtmp = nullptr;
  uint32_t* counts = nullptr;
  unsigned long long *orand = nullptr, *ccnt = nullptr;
  int64_t *c64 = nullptr, *voff = nullptr, *fcnt = nullptr;
  unsigned* flags = nullptr;
  if ((e = scratch.alloc_n(&keys, np)) || (e = scratch.alloc_n(&ktmp, np)) || (e = scratch.alloc_n(&vals, np)) ||
      (e = scratch.alloc_n(&vtmp, np)) || (e = scratch.alloc_n(&counts, (size_t)256 * (np / 4096 + 2))) ||
      (e = scratch.alloc_n(&orand, 2)) || (e = scratch.alloc_n(&ccnt, N)) || (e = scratch.alloc_n(&c64, N)) ||
      (e = scratch.alloc_n(&voff, N + 1)) || (e = scratch.alloc_n(&fcnt, N)) || (e = scratch.alloc_n(&flags, 1)))
    return e;
  if ((e = cudaMemsetAsync(ccnt, 0, sizeof(unsigned long long) * N, st)) ||
      (e = cudaMemsetAsync(flags, 0, sizeof(unsigned), st)))
    return e;
  // the cells' vertex lists in ascending vertex order: a stable sort of
  // (cell, vertex) pairs written in vertex order
  if (nv > 0) {
    k_lz_pairs<<<nb(nv * (d + 1), 256), 256, 0, st>>>(tuples, nv, d, N, keys, vals, ccnt);
    count_launch();
    if ((e = radix_sort_u64(keys, vals, ktmp, vtmp, nv * (d + 1), counts, orand, st))) return e;
  }
  k_lz_u64_to_i64<<<nb(N, 256), 256, 0, st>>>(ccnt, N, c64);
  count_launch();
  if ((e = mc_scan64(c64, N, voff, st))) return e;
  k_lz_facet_list<<<nb(N * 32, 128), 128, 0, st>>>(tuples, d, N, voff, vals, fcnt, nullptr, nullptr, nullptr,
                                                   nullptr, 0);
  count_launch();
  if ((e = out.alloc_n(rowptr, N + 1))) return e;
  if ((e = mc_scan64(fcnt, N, *rowptr, st))) return e;
  if ((e = cudaMemcpyAsync(nnz, *rowptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  const int64_t nn = std::max<int64_t>(*nnz, 1);
  int32_t* erow = nullptr;
  int64_t *m2 = nullptr, *m2off = nullptr;
  double *Vp = nullptr, *Fp = nullptr;
  if ((e = out.alloc_n(V, N)) || (e = out.alloc_n(F, N)) || (e = out.alloc_n(col, nn)) || (e = out.alloc_n(A, nn)) ||
      (e = out.alloc_n(Fd, nn)) || (e = scratch.alloc_n(&erow, nn)) || (e = scratch.alloc_n(&m2, nn)) ||
      (e = scratch.alloc_n(&m2off, nn + 1)) || (e = scratch.alloc_n(&Vp, nn)) || (e = scratch.alloc_n(&Fp, nn)))
    return e;
  k_lz_facet_list<<<nb(N * 32, 128), 128, 0, st>>>(tuples, d, N, voff, vals, nullptr, *rowptr, *col, erow, m2, 1);
  count_launch();
  if ((e = mc_scan64(m2, *nnz, m2off, st))) return e;
  int64_t total2 = 0;
  if ((e = cudaMemcpyAsync(&total2, m2off + *nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  int32_t* lzs = nullptr;
  if ((e = scratch.alloc_n(&lzs, (size_t)std::max<int64_t>((int64_t)(d - 1) * total2, 1)))) return e;
  double fact = 1.0;
  for (int k = 2; k <= d; ++k) fact *= (double)k;
  {  // the walk keeps its per-level state in local memory: make sure the
     // context's per-thread stack holds that frame
    cudaFuncAttributes fa;
    size_t cur = 0;
    if ((e = cudaFuncGetAttributes(&fa, k_lz_facets)) || (e = cudaDeviceGetLimit(&cur, cudaLimitStackSize))) return e;
    const size_t need = (fa.localSizeBytes + 1023) / 1024 * 1024 + 1024;
    if (cur < need && (e = cudaDeviceSetLimit(cudaLimitStackSize, need))) return e;
  }
  // Facets by decreasing vertex count (the first sort's key buffers are
  // free again) when they fill the GPU more than twice over: the walk's long
  // tail then dominates.  Fewer facets keep the CSR order, in which a warp's
  // threads walk one cell's vertices and share their loads in L1.
  int dev = 0, nsm = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lz_facets, 64, 0)))
    return e;
  const int64_t resident = (int64_t)nsm * std::max(occ, 1) * 64;
  int32_t* order = nullptr;
  if (*nnz > 2 * resident) {
    int32_t* otmp = nullptr;
    if ((e = scratch.alloc_n(&order, nn)) || (e = scratch.alloc_n(&otmp, nn))) return e;
    k_lz_order_keys<<<nb(*nnz, 256), 256, 0, st>>>(m2off, *nnz, keys, order);
    count_launch();
    if ((e = radix_sort_u64(keys, order, ktmp, otmp, *nnz, counts, orand, st))) return e;
  }
  k_lz_facet_verts<<<nb(N * 32, 128), 128, 0, st>>>(tuples, d, N, voff, vals, *rowptr, *col, m2off, lzs);
  count_launch();
  unsigned long long* work = nullptr;
  if ((e = scratch.alloc_n(&work, 1)) || (e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), st))) return e;
  const unsigned grid = (unsigned)std::min<int64_t>(nb(*nnz, 64), (int64_t)nsm * std::max(occ, 1));
  k_lz_facets<<<grid, 64, 0, st>>>(X, N, d, tuples, coords, *col, erow, m2off, *nnz, order, lzs, f, fact, Vp, Fp, *A,
                                   *Fd, flags, work);
  count_launch();
  k_lz_cellsum<<<nb(N, 128), 128, 0, st>>>(X, N, d, *rowptr, Vp, Fp, f, *V, *F);
  count_launch();
  if ((e = cudaMemcpyAsync(flags_h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  return cudaGetLastError();
}

}  // namespace vd
