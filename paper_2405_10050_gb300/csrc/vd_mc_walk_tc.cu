// vd_mc_walk_tc.cu -- Monte Carlo RayCast (Section 3.1, Algorithm 3) for
// node sets without candidate lists (high d): a thread block walks the
// node tree once for a tile of 128 rays, and every contraction of that walk
// runs on the tensor cores.
//
// A ray from g = x_i with bound T on its first hit only needs the nodes x_j
// with t_j <= T, i.e. the nodes inside the ball of radius T|u| around
// c = g + T u (t_j <= T  <=>  |x_j - c|^2 <= T^2 |u|^2 for u.(x_j - g) > 0).
//   * Internal tree node with box centre m and radius rho (every node of it
//     lies within rho of m): it can hold such a node only if
//       |m - g|^2 - rho^2 <= 2 T (u.(m - g) + rho |u|),
//     so the 32 children of a popped node are tested for all 128 rays with
//     one MMA (A = ray directions, B = child offsets m - g) plus a few
//     binary32 operations per (ray, child) with directed rounding.  The
//     children any ray needs are pushed on the block's stack, nearest (to g)
//     on top.
//   * Leaf tile of 32 nodes: one MMA gives u.(x_j - g) for every (ray, node)
//     and each thread screens its ray exactly as the list kernels do (an
//     interval of t_j from binary32 bounds, the bound T shrinks, survivors
//     go to a small buffer).
// After the walk each ray rechecks its survivors in binary64 (canonical
// order); rays whose buffer overflowed are finished by the generic kernels.
//
// Ray tiles: with R >= 128 rays per cell a tile is 128 rays of one cell;
// with R = 32 or 64 a tile holds 128 / R cells that are consecutive in the
// tree's Morton order, each with its own B block (w relative to its own g)
// and its own 32 tensor-memory columns.
#include <algorithm>
#include <cmath>

#include "vd_mc_common.cuh"
#include "vd_tc.cuh"

namespace vd {

namespace {

constexpr int kWt = 128;          // threads = rays per tile = MMA M
constexpr int kWtBuf = 8;         // candidates kept per ray
constexpr int kWtStk = kFan * kMaxLev;  // > 1 + 31 (levels - 1): DFS stack bound

struct WalkSmem {
  unsigned char A16[kWt * 32];       // ray directions, fp16, K-major core matrices
  unsigned char B16[kWt * 32];       // up to 4 x 32 rows of offsets
  float r_lo[kWt];                   // leaf: |w|^2 lower bound; internal: |m - g|^2 lower bound
  float r_hi[kWt];                   // leaf: |w|^2 upper bound; internal: rho (rounded up)
  float r_wn[kWt];                   // upper bound of |w|
  int32_t r_id[kWt];                 // leaf: node id or kNoId; internal: child index or -1
  int32_t cb[kWt * kWtBuf];
  float ct[kWt * kWtBuf];
  float den[kWt * 33];
  int32_t stk[kWtStk];
  double g64[4][16];
  int32_t cell[4];
};

__device__ __forceinline__ int wenc(int lev, int64_t idx) { return (lev << 27) | (int)idx; }

// Stages the 32 rows of cell slot `slot` for tree node (lev, idx): offsets
// from g of the 32 leaf nodes (lev 0) or of the 32 children's box centres.
template <int D>
__device__ __forceinline__ void stage_rows(const TreeView& tr, WalkSmem& S, int slot, int lane, int lev, int64_t idx,
                                           float gam, float e1) {
  const int d = tr.d;
  const int row = slot * 32 + lane;
  float w[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) w[k] = 0.f;
  const int32_t cell = S.cell[slot];
  if (lev == 0) {
    const int32_t id = cell == kNoId ? kNoId : tr.ids[idx * kFan + lane];
    if (id != kNoId && id != cell) {
      float ww = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (k < d) {
          w[k] = __double2float_rn(tr.x64[(idx * d + k) * kFan + lane] - S.g64[slot][k]);
          ww = fmaf(w[k], w[k], ww);
        }
      S.r_lo[row] = ww * (1.f - e1);
      S.r_hi[row] = ww * (1.f + e1);
      S.r_wn[row] = sqrtf(ww) * (1.f + gam);
      S.r_id[row] = id;
    } else {
      S.r_id[row] = kNoId;
    }
  } else {
    const int64_t c = idx * kFan + lane;
    if (cell != kNoId && c < tr.cnt[lev - 1]) {
      const int64_t bi = tr.off[lev - 1] + c;
      float ww = 0.f;
      double r2 = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (k < d) {
          const double lo = tr.blo64[k * tr.total + bi], hi = tr.bhi64[k * tr.total + bi];
          const double m = 0.5 * (lo + hi);
          const double h = fmax(m - lo, hi - m);
          r2 = fma(h, h, r2);
          w[k] = __double2float_rn(m - S.g64[slot][k]);
          ww = fmaf(w[k], w[k], ww);
        }
      S.r_lo[row] = ww * (1.f - e1);
      S.r_hi[row] = __double2float_ru(sqrt(r2) * (1.0 + 1e-14));
      S.r_wn[row] = sqrtf(ww) * (1.f + gam);
      S.r_id[row] = (int32_t)c;
    } else {
      S.r_id[row] = -1;
    }
  }
  tc::store_row16(S.B16, row, w);
}

template <int D>
__global__ void __launch_bounds__(kWt) k_mc_walk_tc(TreeView tr, int64_t R, int cpt, uint64_t seed, uint32_t set,
                                                    RayOut ro, Counters* ctr, unsigned long long* work,
                                                    int32_t* fb_cell, int32_t* fb_ray, int64_t fb_cap,
                                                    long long wait_limit) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  WalkSmem& S = *reinterpret_cast<WalkSmem*>(smem_raw);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int64_t s_item;
  __shared__ int s_sp;
  __shared__ uint32_t s_mask;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = tr.d;
  const float gam = (float)(D + 1) * kU32 * 1.01f;
  const float e1 = 1.1f * (gam + 2.1f * kU32);
  const TcBound eb = tc_bound(D);
  const int Rt = cpt > 1 ? (int)R : kWt;               // rays of one cell in a tile
  const int64_t tpc = cpt > 1 ? 1 : (R + kWt - 1) / kWt;  // tiles per cell
  const int64_t nitems = cpt > 1 ? (tr.N + cpt - 1) / cpt : tr.N * tpc;
  const int slot = tid / Rt;
  const uint32_t ncols = 32u * (uint32_t)cpt;
  const uint32_t idesc = tc::idesc_f16_f32(kWt, 32 * cpt);
  int32_t* cb = S.cb + tid * kWtBuf;
  float* ct = S.ct + tid * kWtBuf;
  float* sden = S.den + tid * 33;

  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    s_mask = 0;
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(slot * 32);
  const uint64_t adesc = tc::smem_desc(S.A16, tc::kLbo16, tc::kSbo16);
  const uint64_t bdesc = tc::smem_desc(S.B16, tc::kLbo16, tc::kSbo16);
  uint32_t phase = 0;
  bool timed_out = false;
  unsigned long long n_tiles = 0, n_pairs = 0, n_rech = 0;

  while (!timed_out) {
    if (tid == 0) s_item = (int64_t)atomicAdd(work, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= nitems) break;
    const int64_t q0 = cpt > 1 ? item * cpt : item / tpc;
    const int64_t tb = cpt > 1 ? 0 : item % tpc;
    if (tid < cpt * 16) {
      const int s = tid >> 4, k = tid & 15;
      const int64_t q = q0 + s;
      const int32_t c = q < tr.N ? tr.ids[q] : kNoId;
      S.g64[s][k] = (c != kNoId && k < d) ? tr.X[(int64_t)c * d + k] : 0.0;
      if (k == 0) S.cell[s] = c;
    }
    if (tid == 0) {
      S.stk[0] = wenc(tr.nlev - 1, 0);
      s_sp = 1;
    }
    __syncthreads();
    // ---- this thread's ray ----
    const int32_t cell = S.cell[slot];
    const int64_t k = tb * kWt + (tid % Rt);
    const bool valid = cell != kNoId && k < R;
    double u64[D];
    float u32[D], g32[D], hu[16];
#pragma unroll
    for (int q = 0; q < D; ++q) {
      u64[q] = 0.0;
      g32[q] = __double2float_rn(S.g64[slot][q < 16 ? q : 0]);
    }
    if (valid) mc_direction<D>(seed, set, (uint32_t)cell, (uint32_t)k, d, u64);
#pragma unroll
    for (int q = 0; q < 16; ++q) hu[q] = 0.f;
#pragma unroll
    for (int q = 0; q < D; ++q) {
      u32[q] = __double2float_rn(u64[q]);
      if (q < 16) hu[q] = u32[q];
    }
    tc::store_row16(S.A16, tid, hu);
    float T = INFINITY;
    int nc = 0;
    bool overflow = false;
    if (valid) T = mc_faces<D>(u64, u32, g32, d, cb, ct, nc, kWtBuf, overflow);
    // ---- block walk ----
    while (true) {
      const int sp = s_sp;
      if (sp == 0) break;
      const int e = S.stk[sp - 1];
      const int lev = e >> 27;
      const int64_t idx = e & ((1 << 27) - 1);
      if (warp < cpt) stage_rows<D>(tr, S, warp, lane, lev, idx, gam, e1);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();  // rows staged; everyone has read the stack top
      if (tid == 0) {
        s_sp = sp - 1;
        tc::fence_after_sync();
        tc::mma_f16(tbase, adesc, bdesc, idesc, 0u);
        tc::mma_commit(&mbar);
      }
      const bool ok = tc::mbar_wait(&mbar, phase, wait_limit);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
      tc::fence_after_sync();
      __syncwarp();
      {
        float v[32];
        tc::tmem_ld32(taddr, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) sden[j] = v[j];
      }
      const int r0 = slot * 32;
      if (lev == 0) {
        if (valid) {
          ++n_tiles;
          n_pairs += 32;
#pragma unroll 1
          for (int j = 0; j < 32; ++j) {
            const int32_t id = S.r_id[r0 + j];
            if (id == kNoId) continue;
            const float dj = sden[j];
            const float e = fmaf(eb.a1, S.r_wn[r0 + j], eb.a0);
            const float dh = dj + e;
            const float nlo = S.r_lo[r0 + j];
            if (!(dh > 0.f) || nlo > 2.f * T * dh * (1.f + 8.f * kU32)) continue;
            const float dl = dj - e;
            const float thi = dl > 0.f ? __fdiv_rn(S.r_hi[r0 + j], 2.f * dl) * (1.f + 4.f * kU32) : INFINITY;
            const float tlo = __fdiv_rn(nlo, 2.f * dh) * (1.f - 4.f * kU32);
            if (thi < T) T = thi;
            if (!overflow) overflow = !mc_push(id, tlo, T, cb, ct, nc, kWtBuf);
          }
        }
      } else {
        uint32_t m = 0;
        if (valid) {
          const float T2 = 2.f * T;
#pragma unroll 1
          for (int j = 0; j < 32; ++j) {
            if (S.r_id[r0 + j] < 0) continue;
            const float rho = S.r_hi[r0 + j];
            const float e = fmaf(eb.a1, S.r_wn[r0 + j], eb.a0);
            // |u| <= 1 + 2^-40 after the binary64 normalisation
            const float q = __fadd_ru(__fadd_ru(sden[j], e), __fmul_ru(rho, 1.0000001f));
            const float lhs = __fsub_rd(S.r_lo[r0 + j], __fmul_ru(rho, rho));
            if (!(lhs > __fmul_ru(T2, q))) m |= 1u << j;
          }
        }
        m = __reduce_or_sync(kFull, m);
        if (lane == 0 && m) atomicOr(&s_mask, m);
      }
      tc::fence_before_sync();
      __syncthreads();
      if (lev > 0) {
        if (warp == 0) {
          const uint32_t m = s_mask;
          // nearest child (to the first cell of the tile) on top
          float key = (m >> lane) & 1u ? S.r_lo[lane] : INFINITY;
          int val = lane;
          warp_sort(key, val);
          const int n = __popc(m);
          const int base = s_sp;
          if (lane < n && base + n - 1 - lane < kWtStk)
            S.stk[base + n - 1 - lane] = wenc(lev - 1, idx * kFan + val);
          __syncwarp();
          if (lane == 0) {
            if (base + n > kWtStk) atomicOr(&ctr->flags, kFlagStack);
            s_sp = min(base + n, kWtStk);
            s_mask = 0;
          }
        }
        __syncthreads();
      }
    }
    if (timed_out) break;
    if (valid) {
      if (overflow) {
        const unsigned long long q = atomicAdd(&ctr->fallback, 1ull);
        if ((int64_t)q < fb_cap) {
          fb_cell[q] = cell;
          fb_ray[q] = (int32_t)k;
        } else {
          atomicOr(&ctr->flags, kFlagQueue);
        }
      } else {
        double g64[D];
#pragma unroll
        for (int q = 0; q < D; ++q) g64[q] = q < d ? S.g64[slot][q] : 0.0;
        mc_recheck<D>(tr.X, d, g64, u64, cb, ct, nc, T, ro.hit[(int64_t)cell * R + k],
                      ro.t[(int64_t)cell * R + k], n_rech);
      }
    }
    __syncthreads();  // the next tile rewrites A, g and the stack
  }
  if (timed_out) {
    tc::mbar_wait(&mbar, phase ^ 1u, wait_limit);
    if (tid == 0) atomicOr(&ctr->flags, kFlagTimeout);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
  for (int o = 16; o; o >>= 1) {
    n_tiles += __shfl_xor_sync(kFull, n_tiles, o);
    n_pairs += __shfl_xor_sync(kFull, n_pairs, o);
    n_rech += __shfl_xor_sync(kFull, n_rech, o);
  }
  if (lane == 0) {
    atomicAdd(&ctr->tiles, n_tiles);
    atomicAdd(&ctr->pairs, n_pairs);
    atomicAdd(&ctr->rechecked, n_rech);
  }
}

template <int D>
cudaError_t launch_walk_d(const TreeView& tv, int64_t R, int cpt, uint64_t seed, uint32_t set, const RayOut& ro,
                          Counters* ctr, unsigned long long* work, int32_t* fb_cell, int32_t* fb_ray, int64_t fb_cap,
                          long long wait_limit, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t sm = sizeof(WalkSmem);
  cudaFuncSetAttribute(k_mc_walk_tc<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  // resident blocks from registers, shared memory and warps (the occupancy
  // API reports one block per SM for kernels that allocate tensor memory);
  // tensor memory holds 512 / (32 cpt) blocks
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, k_mc_walk_tc<D>);
  int smem_sm = 0, regs_sm = 0, thr_sm = 0;
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  const int warps = kWt / 32;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  const int by_regs = regs_sm / std::max(1, regs_warp * warps);
  const int by_smem = (int)(smem_sm / (sm + fa.sharedSizeBytes + 1024));
  const int by_thr = thr_sm / kWt;
  const int by_tmem = 16 / cpt;
  const int occ = std::max(1, std::min(std::min(by_regs, by_smem), std::min(by_thr, by_tmem)));
  const int64_t nitems = cpt > 1 ? (tv.N + cpt - 1) / cpt : tv.N * ((R + kWt - 1) / kWt);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * occ, nitems));
  cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
  k_mc_walk_tc<D><<<(unsigned)grid, kWt, sm, st>>>(tv, R, cpt, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap,
                                                    wait_limit);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

// All N*R MC rays of the node set by the block tree walk with tensor-core
// screening; rays whose candidate buffer overflowed are finished by
// launch_raycast.  Same contract as launch_mc_cells.
cudaError_t launch_mc_walk_tc(const TreeView& tv, int64_t R, uint64_t seed, uint32_t set, const RayOut& ro,
                              Counters* ctr, long long wait_limit, cudaStream_t st, int64_t* nfallback) {
  unsigned long long* work = reinterpret_cast<unsigned long long*>(&ctr->aux1);
  int32_t* fb_cell = ro.fallback_list;
  int32_t* fb_ray = ro.fallback_list + ro.fallback_cap / 2;
  const int64_t fb_cap = ro.fallback_cap / 2;
  const int cpt = (R < kWt && R % 32 == 0) ? (int)(kWt / R) : 1;
  const long long wl = wait_limit > 0 ? wait_limit : (1ll << 22);
  cudaMemsetAsync(&ctr->fallback, 0, sizeof(unsigned long long), st);
  cudaError_t e;
#define VD_WALK(DD) launch_walk_d<DD>(tv, R, cpt, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wl, st)
  switch (tv.d) {
    case 1: e = VD_WALK(1); break;
    case 2: e = VD_WALK(2); break;
    case 3: e = VD_WALK(3); break;
    case 4: e = VD_WALK(4); break;
    case 5: e = VD_WALK(5); break;
    case 6: e = VD_WALK(6); break;
    case 7:
    case 8: e = VD_WALK(8); break;
    case 9: case 10: case 11: case 12: e = VD_WALK(12); break;
    default: e = VD_WALK(16); break;
  }
#undef VD_WALK
  if (e != cudaSuccess) return e;
  unsigned long long nfb = 0;
  cudaMemcpyAsync(&nfb, &ctr->fallback, sizeof(nfb), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  const int64_t n = std::min<int64_t>((int64_t)nfb, fb_cap);
  if (nfallback) *nfallback += n;
  if (n == 0) return cudaSuccess;
  RaySource rs;
  rs.mode = 1;
  rs.R = n;
  rs.mc_cell = fb_cell;
  rs.mc_ray = fb_ray;
  rs.mc_rpc = R;
  rs.seed = seed;
  rs.set = set;
  rs.box = 1;
  RayOut r2 = ro;
  r2.fallback_list = nullptr;
  r2.fallback_cap = 0;
  TreeView tv2 = tv;
  tv2.K = 0;
  return launch_raycast(tv2, rs, r2, VD_FP32, ctr, st, nullptr);
}

}  // namespace vd
