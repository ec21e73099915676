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
constexpr int kGroups = 4;        // 32-row B groups (32 tensor-memory columns each) per round
constexpr int kWtStk = kFan * kMaxLev * kGroups;  // stack bound for rounds of up to kGroups entries

struct WalkSmem {
  unsigned char A16[kWt * 32];       // ray directions, fp16, K-major core matrices
  unsigned char B16[kWt * 32];       // kGroups x 32 rows of offsets
  // per staged row, x = threshold, y = additive term of the test against den = u.w:
  //   leaf (node j):  x = lower bound of |w|^2 (+inf if absent), y = error bound of den;
  //                   t_j <= T possible iff den + y > 0 and x <= 2 T (den + y) (1 + 8u)
  //   internal child: x = |m - g|^2 - rho^2 rounded down (+inf if absent),
  //                   y = err(den) + rho rounded up; needed iff x <= 2 T (den + y)
  float2 r_ae[kWt];
  float r_hi[kWt];                   // leaf: |w|^2 upper bound; internal: |m - g|^2 (sort key)
  int32_t r_id[kWt];                 // leaf: node id or kNoId
  float e_w[kGroups][16];            // popped entry's own box: centre - g (binary32)
  float e_lo[kGroups], e_rho[kGroups], e_wn[kGroups];
  int32_t cb[kWt * kWtBuf];
  float ct[kWt * kWtBuf];
  float den[kWt * 33];
  int32_t stk[kWtStk];
  int32_t ent[kGroups];              // entries popped this round
  uint32_t mask[kGroups];            // children wanted by any ray, per popped internal entry
  double g64[4][16];
  float g32[4][16];
  int32_t cell[4];
};

__device__ __forceinline__ int wenc(int lev, int64_t idx) { return (lev << 27) | (int)idx; }

// Binary32 error model of the staged offsets: each component of
// w32 = fl(x32 - g32) is within EW of the exact x - g (x32, g32 the nearest
// binary32 of x and g), ww32 = fma chain of w32^2 within gamma_D of |w32|^2.
struct WalkEps {
  float gam;   // gamma_D of the fma chains
  float EW;    // per-component absolute error of w32
  float eabs;  // sqrt(D) EW (1.01): |u.(w32 - w)| for |u| <= 1
  float a1, a0;  // MMA den: |den - u.w| <= a1 |w32| + a0 (a0 includes eabs)
};

// Upper bound of the exact |w|^2 from ww32.
__device__ __forceinline__ float d2_upper(float ww, const WalkEps& ep) {
  const float t = sqrtf(ww) * (1.f + ep.gam) + ep.eabs;
  return t * t * (1.f + 4.f * kU32);
}

// Stages the 32 rows of group grp (cell slot `slot`) for tree node
// (lev, idx): offsets from g of the 32 leaf nodes (lev 0) or of the 32
// children's box centres, and the node's own box (centre offset, radius).
// All in binary32 with directed rounding where a bound is formed.
template <int D>
__device__ __forceinline__ void stage_rows(const TreeView& tr, WalkSmem& S, int grp, int slot, int lane, int lev,
                                           int64_t idx, const WalkEps& ep) {
  const int d = tr.d;
  const int row = grp * 32 + lane;
  {  // the node's own box, one dimension per lane
    const int64_t bi = tr.off[lev] + idx;
    float w = 0.f, h2 = 0.f;
    if (lane < d) {
      const float lo = tr.blo32[lane * tr.total + bi], hi = tr.bhi32[lane * tr.total + bi];
      const float m = 0.5f * (lo + hi);
      const float h = fmaxf(__fsub_ru(m, lo), __fsub_ru(hi, m));
      h2 = __fmul_ru(h, h);
      w = m - S.g32[slot][lane];
    }
    float ww = w * w;
    for (int o = 16; o; o >>= 1) {
      ww += __shfl_xor_sync(kFull, ww, o);
      h2 = __fadd_ru(h2, __shfl_xor_sync(kFull, h2, o));
    }
    if (lane < 16) S.e_w[grp][lane] = w;
    if (lane == 0) {
      S.e_lo[grp] = true_d2_lower(ww, ep.gam, ep.EW, D);
      S.e_rho[grp] = tr.rho32 ? fminf(__fsqrt_ru(h2), tr.rho32[bi]) : __fsqrt_ru(h2);
      S.e_wn[grp] = sqrtf(ww) * (1.f + ep.gam);
    }
  }
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
          w[k] = tr.x32[(idx * d + k) * kFan + lane] - S.g32[slot][k];
          ww = fmaf(w[k], w[k], ww);
        }
      S.r_ae[row] = make_float2(true_d2_lower(ww, ep.gam, ep.EW, D), fmaf(ep.a1, sqrtf(ww) * (1.f + ep.gam), ep.a0));
      S.r_hi[row] = d2_upper(ww, ep);
      S.r_id[row] = id;
    } else {
      S.r_ae[row] = make_float2(INFINITY, 1.f);
      S.r_id[row] = kNoId;
    }
  } else {
    const int64_t c = idx * kFan + lane;
    if (cell != kNoId && c < tr.cnt[lev - 1]) {
      const int64_t bi = tr.off[lev - 1] + c;
      float ww = 0.f, r2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (k < d) {
          const float lo = tr.blo32[k * tr.total + bi], hi = tr.bhi32[k * tr.total + bi];
          const float m = 0.5f * (lo + hi);
          const float h = fmaxf(__fsub_ru(m, lo), __fsub_ru(hi, m));
          r2 = __fmaf_ru(h, h, r2);
          w[k] = m - S.g32[slot][k];
          ww = fmaf(w[k], w[k], ww);
        }
      const float d2lo = true_d2_lower(ww, ep.gam, ep.EW, D);
      const float rho = tr.rho32 ? fminf(__fsqrt_ru(r2), tr.rho32[bi]) : __fsqrt_ru(r2);
      const float err = fmaf(ep.a1, sqrtf(ww) * (1.f + ep.gam), ep.a0);
      // |u| <= 1 + 2^-40 after the binary64 normalisation
      S.r_ae[row] = make_float2(__fsub_rd(d2lo, __fmul_ru(rho, rho)), __fadd_ru(err, __fmul_ru(rho, 1.0000001f)));
      S.r_hi[row] = d2lo;
    } else {
      S.r_ae[row] = make_float2(INFINITY, 0.f);
      S.r_hi[row] = INFINITY;
    }
  }
  tc::store_row16(S.B16, row, w);
}

template <int D>
__global__ void __launch_bounds__(kWt, 4) k_mc_walk_tc(TreeView tr, int64_t R, int cpt, uint64_t seed, uint32_t set,
                                                    RayOut ro, Counters* ctr, unsigned long long* work,
                                                    int32_t* fb_cell, int32_t* fb_ray, int64_t fb_cap,
                                                    long long wait_limit) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  WalkSmem& S = *reinterpret_cast<WalkSmem*>(smem_raw);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int64_t s_item;
  __shared__ int s_sp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = tr.d;
  WalkEps ep;
  ep.gam = (float)(D + 1) * kU32 * 1.01f;
  ep.EW = 4.01f * kU32 * tr.coord_abs;
  ep.eabs = sqrtf((float)D) * ep.EW * 1.01f;
  const float gam = ep.gam;
  {
    const TcBound eb = tc_bound(D);
    ep.a1 = eb.a1;
    ep.a0 = eb.a0 + ep.eabs;
  }
  const int Rt = cpt > 1 ? (int)R : kWt;               // rays of one cell in a tile
  const int64_t tpc = cpt > 1 ? 1 : (R + kWt - 1) / kWt;  // tiles per cell
  const int64_t nitems = cpt > 1 ? (tr.N + cpt - 1) / cpt : tr.N * tpc;
  const int slot = tid / Rt;
  const int P = kGroups / cpt;  // entries per round
  const uint32_t ncols = 32u * kGroups;
  const float a1f = 1.1f * (gam + 2.1f * kU32);  // binary32 dot product of u and w: error <= a1f |w|
  int32_t* cb = S.cb + tid * kWtBuf;
  float* ct = S.ct + tid * kWtBuf;
  float* sden = S.den + tid * 33;

  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);
  if (tid < kGroups) S.mask[tid] = 0;
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16);
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
      const double gk = (c != kNoId && k < d) ? tr.X[(int64_t)c * d + k] : 0.0;
      S.g64[s][k] = gk;
      S.g32[s][k] = __double2float_rn(gk);
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
      g32[q] = S.g32[slot][q];
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
    // ---- block walk: each round pops up to P entries ----
    while (true) {
      const int sp = s_sp;
      if (sp == 0) break;
      const int np = min(P, sp);
      if (warp < np * cpt) {
        const int e = S.stk[sp - 1 - warp / cpt];
        if (lane == 0 && warp % cpt == 0) S.ent[warp / cpt] = e;
        stage_rows<D>(tr, S, warp, warp % cpt, lane, e >> 27, e & ((1 << 27) - 1), ep);
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();  // rows staged; everyone has read the stack
      if (tid == 0) {
        s_sp = sp - np;
        tc::fence_after_sync();
        tc::mma_f16(tbase, adesc, bdesc, tc::idesc_f16_f32(kWt, 32 * np * cpt), 0u);
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
      for (int p = 0; p < np; ++p) {
        const int grp = p * cpt + slot;
        const int r0 = grp * 32;
        const int e = S.ent[p];
        float v[32];
        tc::tmem_ld32(taddr + (uint32_t)(grp * 32), v);
        // does this ray still need the entry?  ball of T around g + T u
        // against the sphere of the entry's own box, binary32 dot product
        bool need = valid;
        if (need) {
          float sdot = 0.f;
#pragma unroll
          for (int q = 0; q < D; ++q) sdot = fmaf(u32[q], S.e_w[grp][q], sdot);
          const float rho = S.e_rho[grp];
          const float qv = __fadd_ru(__fadd_ru(sdot, fmaf(a1f, S.e_wn[grp], ep.eabs)), __fmul_ru(rho, 1.0000001f));
          const float lhs = __fsub_rd(S.e_lo[grp], __fmul_ru(rho, rho));
          need = !(lhs > __fmul_ru(2.f * T, qv));
        }
        if ((e >> 27) == 0) {
          uint32_t pass = 0;
          if (need) {
            ++n_tiles;
            n_pairs += 32;
            const float T2u = 2.f * T * (1.f + 10.f * kU32);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float2 ae = S.r_ae[r0 + j];
              const float dh = v[j] + ae.y;
              if (dh > 0.f && !(ae.x > T2u * dh)) pass |= 1u << j;
            }
          }
          if (pass) {  // rare: exact interval test with the current bound
#pragma unroll
            for (int j = 0; j < 32; ++j) sden[j] = v[j];
            while (pass) {
              const int j = __ffs(pass) - 1;
              pass &= pass - 1;
              const float2 ae = S.r_ae[r0 + j];
              const float dj = sden[j];
              const float dh = dj + ae.y;
              if (ae.x > 2.f * T * dh * (1.f + 8.f * kU32)) continue;
              const float dl = dj - ae.y;
              const float thi = dl > 0.f ? __fdiv_rn(S.r_hi[r0 + j], 2.f * dl) * (1.f + 4.f * kU32) : INFINITY;
              const float tlo = __fdiv_rn(ae.x, 2.f * dh) * (1.f - 4.f * kU32);
              if (thi < T) T = thi;
              if (!overflow) overflow = !mc_push(S.r_id[r0 + j], tlo, T, cb, ct, nc, kWtBuf);
            }
          }
        } else {
          uint32_t m = 0;
          if (need) {
            const float T2 = 2.f * T;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float2 ae = S.r_ae[r0 + j];
              if (!(ae.x > __fmul_ru(T2, __fadd_ru(v[j], ae.y)))) m |= 1u << j;
            }
          }
          m = __reduce_or_sync(kFull, m);
          if (lane == 0 && m) atomicOr(&S.mask[p], m);
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      if (warp == 0) {
        // children of the popped internal entries, the first entry's on top,
        // each entry's children nearest (to the tile's first cell) on top
        for (int p = np - 1; p >= 0; --p) {
          const int e = S.ent[p];
          if ((e >> 27) == 0) continue;
          const uint32_t m = S.mask[p];
          float key = (m >> lane) & 1u ? S.r_hi[p * cpt * 32 + lane] : INFINITY;
          int val = lane;
          warp_sort(key, val);
          const int n = __popc(m);
          const int base = s_sp;
          if (lane < n && base + n - 1 - lane < kWtStk)
            S.stk[base + n - 1 - lane] = wenc((e >> 27) - 1, (int64_t)(e & ((1 << 27) - 1)) * kFan + val);
          __syncwarp();
          if (lane == 0) {
            if (base + n > kWtStk) atomicOr(&ctr->flags, kFlagStack);
            s_sp = min(base + n, kWtStk);
            S.mask[p] = 0;
          }
          __syncwarp();
        }
      }
      __syncthreads();
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
        ro.t[(int64_t)cell * R + k] = (double)T;  // the bound found so far seeds the tree walk
      } else {
        double g64[D], uu[D];
#pragma unroll
        for (int q = 0; q < D; ++q) g64[q] = q < d ? S.g64[slot][q] : 0.0;
        mc_direction<D>(seed, set, (uint32_t)cell, (uint32_t)k, d, uu);  // drawn again: same bits
        mc_recheck<D>(tr.X, d, g64, uu, cb, ct, nc, T, ro.hit[(int64_t)cell * R + k],
                      ro.t[(int64_t)cell * R + k], n_rech);
      }
    }
    __syncthreads();  // the next tile rewrites A, g and the stack
  }
  if (timed_out) {
    // the MMA still in flight must finish before its tensor memory is freed:
    // this wait has its own generous bound, whatever limit gave up above
    tc::mbar_wait(&mbar, phase ^ 1u, wait_limit > (1ll << 24) ? wait_limit : (1ll << 24));
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
  allow_max_dyn_smem(k_mc_walk_tc<D>);
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
  const int by_tmem = 512 / (32 * kGroups);
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
  const long long wl = wait_polls(wait_limit);
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
  rs.t_hint = 1;
  RayOut r2 = ro;
  r2.fallback_list = nullptr;
  r2.fallback_cap = 0;
  TreeView tv2 = tv;
  tv2.K = 0;
  return launch_raycast(tv2, rs, r2, VD_FP32, ctr, st, nullptr);
}

}  // namespace vd
