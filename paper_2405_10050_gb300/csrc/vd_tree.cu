// vd_tree.cu -- node preparation: Morton codes, a stable LSD radix sort,
// 32-node leaf tiles (binary64 and binary32 copies, SoA per tile) and a
// 32-way bounding-box hierarchy over the tiles.  The hierarchy replaces the
// nearest-neighbour structure that the RayCast of Section 2.2 (Algorithm 1,
// nn) relies on: a tile is visited only if its box meets the current ball.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "vd_dev.cuh"

namespace vd {

namespace {

constexpr int kRsThreads = 256;
constexpr int kRsSub = 16;                       // sub-chunks of 256 keys per block
constexpr int kRsChunk = kRsThreads * kRsSub;    // keys per block

__global__ void k_bounds_partial(const double* X, int64_t N, int d, double* part) {
  __shared__ double slo[kRsThreads], shi[kRsThreads];
  for (int k = 0; k < d; ++k) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
      const double x = X[i * d + k];
      if (isfinite(x)) {
        lo = fmin(lo, x);
        hi = fmax(hi, x);
      } else {  // NaN or infinity: infinite bounds, which the host reports
        lo = -INFINITY;
        hi = INFINITY;
      }
    }
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
        shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      part[(int64_t)blockIdx.x * 2 * d + k] = slo[0];
      part[(int64_t)blockIdx.x * 2 * d + d + k] = shi[0];
    }
    __syncthreads();
  }
}

__global__ void k_bounds_final(const double* part, int nblk, int d, double* out) {
  const int k = threadIdx.x;
  if (k >= d) return;
  double lo = INFINITY, hi = -INFINITY;
  for (int b = 0; b < nblk; ++b) {
    lo = fmin(lo, part[(int64_t)b * 2 * d + k]);
    hi = fmax(hi, part[(int64_t)b * 2 * d + d + k]);
  }
  out[k] = lo;
  out[d + k] = hi;
}

__global__ void k_morton(const double* X, int64_t N, int d, const double* bounds, uint64_t* keys, int32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int b = min(64 / d, 32);
  uint32_t q[VD_MAX_D];
  for (int k = 0; k < d; ++k) {
    const double lo = bounds[k], hi = bounds[d + k];
    const double span = hi - lo;
    double f = span > 0 ? (X[i * d + k] - lo) / span : 0.0;
    f = fmin(fmax(f, 0.0), 1.0);
    const double lim = ldexp(1.0, b) - 1.0;
    q[k] = (uint32_t)fmin(floor(f * ldexp(1.0, b)), lim);
  }
  uint64_t code = 0;
  for (int L = b - 1; L >= 0; --L)
    for (int k = 0; k < d; ++k) code = (code << 1) | ((q[k] >> L) & 1u);
  keys[i] = code;
  vals[i] = (int32_t)i;
}

__global__ void k_rs_hist(const uint64_t* keys, int64_t n, int shift, uint32_t* counts, int nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsChunk;
  for (int i = threadIdx.x; i < kRsChunk; i += kRsThreads) {
    const int64_t idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `total` counts in place, in two launches of P <= 256
// blocks of 1024 threads: block b owns the tile [b tile, (b+1) tile); the
// first launch writes each tile's sum to part[b], the second scans its tile
// (1024 values at a time, coalesced) from the sum of the tiles before it.
constexpr int kScanThreads = 1024;

__global__ void k_rs_scan_reduce(const uint32_t* counts, int64_t total, int64_t tile, uint32_t* part) {
  __shared__ uint32_t ws[kScanThreads / 32];
  const int64_t b0 = blockIdx.x * tile, b1 = min(total, b0 + tile);
  uint32_t s = 0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += kScanThreads) s += counts[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = ws[threadIdx.x];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

__global__ void k_rs_scan_tiles(uint32_t* counts, int64_t total, int64_t tile, const uint32_t* part) {
  __shared__ uint32_t ws[kScanThreads / 32];
  __shared__ uint32_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    uint32_t c = 0;
    for (unsigned b = 0; b < blockIdx.x; ++b) c += part[b];
    carry = c;
  }
  __syncthreads();
  const int64_t b0 = blockIdx.x * tile, b1 = min(total, b0 + tile);
  for (int64_t base = b0; base < b1; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const uint32_t x = i < b1 ? counts[i] : 0u;
    uint32_t v = x;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) ws[warp] = v;
    __syncthreads();
    if (warp == 0) {  // scan of the warp totals
      uint32_t t = ws[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, t, o);
        if (lane >= o) t += y;
      }
      ws[lane] = t;
    }
    __syncthreads();
    const uint32_t before = carry + (warp > 0 ? ws[warp - 1] : 0u) + v - x;
    if (i < b1) counts[i] = before;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = before + x;
    __syncthreads();
  }
}

// Stable scatter: keys keep their input order within a digit.
__global__ void k_rs_scatter(const uint64_t* kin, const int32_t* vin, uint64_t* kout, int32_t* vout, int64_t n,
                             int shift, const uint32_t* offs, int nblk) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wc[kRsThreads / 32][257];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kRsChunk;
  const unsigned lt = (1u << lane) - 1u;
  for (int sub = 0; sub < kRsSub; ++sub) {
    const int64_t idx = base + (int64_t)sub * kRsThreads + tid;
    const bool valid = idx < n;
    uint64_t key = 0;
    int32_t val = 0;
    unsigned dig = 256;
    if (valid) {
      key = kin[idx];
      val = vin[idx];
      dig = (unsigned)((key >> shift) & 255u);
    }
    for (int j = tid; j < (kRsThreads / 32) * 257; j += kRsThreads) (&wc[0][0])[j] = 0;
    __syncthreads();
    const unsigned mask = __match_any_sync(kFull, dig);
    const unsigned rank = __popc(mask & lt);
    if (valid && rank == 0) wc[warp][dig] = __popc(mask);
    __syncthreads();
    {
      uint32_t r = run[tid];
      for (int w = 0; w < kRsThreads / 32; ++w) {
        const uint32_t c = wc[w][tid];
        wc[w][tid] = r;
        r += c;
      }
      run[tid] = r;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wc[warp][dig] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

__global__ void k_key_span(const uint64_t* keys, int64_t n, unsigned long long* orand) {
  unsigned long long o = 0, a = ~0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    o |= keys[i];
    a &= keys[i];
  }
  for (int s = 16; s; s >>= 1) {
    o |= __shfl_xor_sync(kFull, o, s);
    a &= __shfl_xor_sync(kFull, a, s);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicOr(&orand[0], o);
    atomicAnd(&orand[1], a);
  }
}

__global__ void k_tiles(const double* X, int64_t N, int d, const int32_t* order, int64_t ntiles, double* x64,
                        float* x32, int32_t* ids) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ntiles * kTile) return;
  const int64_t tile = p / kTile;
  const int lane = (int)(p % kTile);
  const bool valid = p < N;
  const int32_t id = valid ? order[p] : order[tile * kTile];  // pads copy the tile's first node
  for (int k = 0; k < d; ++k) {
    const double x = X[(int64_t)id * d + k];
    x64[(tile * d + k) * kTile + lane] = x;
    x32[(tile * d + k) * kTile + lane] = __double2float_rn(x);
  }
  ids[p] = valid ? id : kNoId;
}

__global__ void k_leaf_bbox(const double* x64, int64_t ntiles, int d, int64_t total, int64_t off, double* lo64,
                            double* hi64, float* lo32, float* hi32) {
  const int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (tile >= ntiles) return;
  for (int k = 0; k < d; ++k) {
    const double x = x64[(tile * d + k) * kTile + lane];  // pads duplicate a valid node
    double lo = x, hi = x;
    for (int s = 16; s; s >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(kFull, lo, s));
      hi = fmax(hi, __shfl_xor_sync(kFull, hi, s));
    }
    if (lane == 0) {
      lo64[k * total + off + tile] = lo;
      hi64[k * total + off + tile] = hi;
      lo32[k * total + off + tile] = f32_down(lo);
      hi32[k * total + off + tile] = f32_up(hi);
    }
  }
}

__global__ void k_level_bbox(int d, int64_t total, int64_t off_child, int64_t n_child, int64_t off_par,
                             int64_t n_par, double* lo64, double* hi64, float* lo32, float* hi32) {
  const int64_t par = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (par >= n_par) return;
  const int64_t c = par * kFan + lane;
  const bool valid = c < n_child;
  for (int k = 0; k < d; ++k) {
    double lo = valid ? lo64[k * total + off_child + c] : INFINITY;
    double hi = valid ? hi64[k * total + off_child + c] : -INFINITY;
    for (int s = 16; s; s >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(kFull, lo, s));
      hi = fmax(hi, __shfl_xor_sync(kFull, hi, s));
    }
    if (lane == 0) {
      lo64[k * total + off_par + par] = lo;
      hi64[k * total + off_par + par] = hi;
      lo32[k * total + off_par + par] = f32_down(lo);
      hi32[k * total + off_par + par] = f32_up(hi);
    }
  }
}

// Radius of each node's points around the binary32 centre of its box,
// m = 0.5 (lo32 + hi32) rounded to nearest in binary32 (the centre the
// tensor-core walk uses), rounded up: leaves from their points, parents as
// max over children of |m_child - m| + rho_child.  In high d the points of a
// box stay far from its corners, so this radius is well below the box's
// half-diagonal.
__global__ void k_leaf_rho(const double* x64, int64_t ntiles, int d, int64_t total, int64_t off, const float* lo32,
                           const float* hi32, float* rho) {
  const int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (tile >= ntiles) return;
  double r2 = 0.0;
  for (int k = 0; k < d; ++k) {
    const float m = 0.5f * (lo32[k * total + off + tile] + hi32[k * total + off + tile]);
    const double w = x64[(tile * d + k) * kTile + lane] - (double)m;  // pads duplicate a valid node
    r2 = fma(w, w, r2);
  }
  for (int s = 16; s; s >>= 1) r2 = fmax(r2, __shfl_xor_sync(kFull, r2, s));
  if (lane == 0) rho[off + tile] = f32_up(sqrt(r2) * (1.0 + 1e-14));
}

__global__ void k_level_rho(int d, int64_t total, int64_t off_child, int64_t n_child, int64_t off_par, int64_t n_par,
                            const float* lo32, const float* hi32, float* rho) {
  const int64_t par = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (par >= n_par) return;
  const int64_t c = par * kFan + lane;
  double r = 0.0;
  if (c < n_child) {
    double q2 = 0.0;
    for (int k = 0; k < d; ++k) {
      const float mp = 0.5f * (lo32[k * total + off_par + par] + hi32[k * total + off_par + par]);
      const float mc = 0.5f * (lo32[k * total + off_child + c] + hi32[k * total + off_child + c]);
      const double w = (double)mc - (double)mp;
      q2 = fma(w, w, q2);
    }
    r = sqrt(q2) * (1.0 + 1e-14) + (double)rho[off_child + c];
  }
  for (int s = 16; s; s >>= 1) r = fmax(r, __shfl_xor_sync(kFull, r, s));
  if (lane == 0) rho[off_par + par] = f32_up(r * (1.0 + 1e-14));
}

inline int nblocks(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

// Sorts (keys, vals) in place by key, stably; tmp buffers of the same sizes;
// counts holds 256 (ceil(n / 4096) + 1) values (the digit counts of every
// 4096-key block, then the scan's tile sums).
cudaError_t radix_sort_u64(uint64_t* keys, int32_t* vals, uint64_t* ktmp, int32_t* vtmp, int64_t n,
                           uint32_t* counts, unsigned long long* orand, cudaStream_t st) {
  static_assert(kRsChunk == 4096, "callers size counts for 4096-key blocks");
  if (n <= 1) return cudaSuccess;
  const int nblk = nblocks(n, kRsChunk);
  const int64_t total = (int64_t)256 * nblk;
  const int nscan = (int)std::min<int64_t>(256, (total + kScanThreads - 1) / kScanThreads);
  const int64_t tile = (total + nscan - 1) / nscan;
  uint32_t* part = counts + total;
  unsigned long long init[2] = {0ull, ~0ull};
  cudaMemcpyAsync(orand, init, sizeof(init), cudaMemcpyHostToDevice, st);
  k_key_span<<<std::min(nblocks(n, 256), 1024), 256, 0, st>>>(keys, n, orand); count_launch();
  unsigned long long oa[2];
  cudaMemcpyAsync(oa, orand, sizeof(oa), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  const unsigned long long varying = oa[0] ^ oa[1];
  uint64_t* ka = keys;
  int32_t* va = vals;
  uint64_t* kb = ktmp;
  int32_t* vb = vtmp;
  for (int shift = 0; shift < 64; shift += 8) {
    if (((varying >> shift) & 255ull) == 0) continue;
    k_rs_hist<<<nblk, kRsThreads, 0, st>>>(ka, n, shift, counts, nblk); count_launch();
    k_rs_scan_reduce<<<nscan, kScanThreads, 0, st>>>(counts, total, tile, part); count_launch();
    k_rs_scan_tiles<<<nscan, kScanThreads, 0, st>>>(counts, total, tile, part); count_launch();
    k_rs_scatter<<<nblk, kRsThreads, 0, st>>>(ka, va, kb, vb, n, shift, counts, nblk); count_launch();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  }
  return cudaGetLastError();
}

cudaError_t build_tree(const double* X, int64_t N, int d, cudaStream_t st, DevBufs& bufs, TreeView* tv) {
  cudaError_t e;
#define VD_TRY(x)                  \
  do {                             \
    e = (x);                       \
    if (e != cudaSuccess) return e; \
  } while (0)
  TreeView t;
  t.d = d;
  t.N = N;
  t.X = X;
  t.ntiles = (N + kTile - 1) / kTile;
  // level sizes
  int64_t c = t.ntiles;
  t.nlev = 0;
  while (true) {
    t.cnt[t.nlev] = c;
    t.off[t.nlev] = t.total;
    t.total += c;
    ++t.nlev;
    if (c == 1) break;
    c = (c + kFan - 1) / kFan;
    if (t.nlev >= kMaxLev) return cudaErrorInvalidValue;
  }
  // scratch (freed at the end)
  DevBufs scratch;
  scratch.arena = bufs.arena;
  const int nb_bounds = std::min(nblocks(N, 256), 256);
  double *part = nullptr, *bounds = nullptr;
  uint64_t *keys = nullptr, *ktmp = nullptr;
  int32_t *vals = nullptr, *vtmp = nullptr;
  uint32_t* counts = nullptr;
  unsigned long long* orand = nullptr;
  const int nblk = nblocks(N, kRsChunk);
  if ((e = scratch.alloc_n(&part, (size_t)nb_bounds * 2 * d)) != cudaSuccess ||
      (e = scratch.alloc_n(&bounds, 2 * d)) != cudaSuccess || (e = scratch.alloc_n(&keys, N)) != cudaSuccess ||
      (e = scratch.alloc_n(&ktmp, N)) != cudaSuccess || (e = scratch.alloc_n(&vals, N)) != cudaSuccess ||
      (e = scratch.alloc_n(&vtmp, N)) != cudaSuccess ||
      (e = scratch.alloc_n(&counts, (size_t)256 * (nblk + 1))) != cudaSuccess ||
      (e = scratch.alloc_n(&orand, 2)) != cudaSuccess) {
    scratch.release();
    return e;
  }
  k_bounds_partial<<<nb_bounds, 256, 0, st>>>(X, N, d, part); count_launch();
  k_bounds_final<<<1, 32, 0, st>>>(part, nb_bounds, d, bounds); count_launch();
  double hb[2 * VD_MAX_D];
  cudaMemcpyAsync(hb, bounds, sizeof(double) * 2 * d, cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { scratch.release(); return e; }
  double ca = 1.0;
  for (int k = 0; k < 2 * d; ++k) ca = std::max(ca, std::fabs(hb[k]));
  for (int k = 0; k < d; ++k) {
    t.box_lo[k] = hb[k];
    t.box_hi[k] = hb[d + k];
  }
  if (!std::isfinite(ca)) { scratch.release(); return cudaErrorInvalidValue; }
  t.coord_abs = (float)ca * (1.0f + 1e-6f);
  k_morton<<<nblocks(N, 256), 256, 0, st>>>(X, N, d, bounds, keys, vals); count_launch();
  e = radix_sort_u64(keys, vals, ktmp, vtmp, N, counts, orand, st);
  if (e != cudaSuccess) { scratch.release(); return e; }
  double *x64 = nullptr, *lo64 = nullptr, *hi64 = nullptr;
  float *x32 = nullptr, *lo32 = nullptr, *hi32 = nullptr, *rho32 = nullptr;
  int32_t* ids = nullptr;
  if ((e = bufs.alloc_n(&x64, (size_t)t.ntiles * d * kTile)) != cudaSuccess ||
      (e = bufs.alloc_n(&x32, (size_t)t.ntiles * d * kTile)) != cudaSuccess ||
      (e = bufs.alloc_n(&ids, (size_t)t.ntiles * kTile)) != cudaSuccess ||
      (e = bufs.alloc_n(&lo64, (size_t)t.total * d)) != cudaSuccess ||
      (e = bufs.alloc_n(&hi64, (size_t)t.total * d)) != cudaSuccess ||
      (e = bufs.alloc_n(&lo32, (size_t)t.total * d)) != cudaSuccess ||
      (e = bufs.alloc_n(&hi32, (size_t)t.total * d)) != cudaSuccess ||
      (e = bufs.alloc_n(&rho32, (size_t)t.total)) != cudaSuccess) {
    scratch.release();
    return e;
  }
  k_tiles<<<nblocks(t.ntiles * kTile, 256), 256, 0, st>>>(X, N, d, vals, t.ntiles, x64, x32, ids); count_launch();
  k_leaf_bbox<<<nblocks(t.ntiles * 32, 256), 256, 0, st>>>(x64, t.ntiles, d, t.total, t.off[0], lo64, hi64, lo32,
                                                             hi32); count_launch();
  for (int L = 1; L < t.nlev; ++L)
    k_level_bbox<<<nblocks(t.cnt[L] * 32, 256), 256, 0, st>>>(d, t.total, t.off[L - 1], t.cnt[L - 1], t.off[L],
                                                                t.cnt[L], lo64, hi64, lo32, hi32); count_launch();
  k_leaf_rho<<<nblocks(t.ntiles * 32, 256), 256, 0, st>>>(x64, t.ntiles, d, t.total, t.off[0], lo32, hi32, rho32);
  count_launch();
  for (int L = 1; L < t.nlev; ++L) {
    k_level_rho<<<nblocks(t.cnt[L] * 32, 256), 256, 0, st>>>(d, t.total, t.off[L - 1], t.cnt[L - 1], t.off[L],
                                                               t.cnt[L], lo32, hi32, rho32);
    count_launch();
  }
  e = cudaStreamSynchronize(st);
  bufs.requested += scratch.requested;  // the scratch was carved from the same block: size it for both
  scratch.release();
  if (e != cudaSuccess) return e;
  VD_TRY(cudaGetLastError());
  t.x64 = x64;
  t.x32 = x32;
  t.ids = ids;
  t.blo64 = lo64;
  t.bhi64 = hi64;
  t.blo32 = lo32;
  t.bhi32 = hi32;
  t.rho32 = rho32;
  *tv = t;
  return cudaSuccess;
#undef VD_TRY
}

}  // namespace vd
