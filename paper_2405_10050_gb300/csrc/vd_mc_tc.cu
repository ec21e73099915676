// vd_mc_tc.cu -- cell-centric Monte Carlo RayCast with the u.w contraction
// on the tensor cores (tcgen05).  Same method as vd_mc_cell.cu (Section 3.1,
// Algorithm 3; candidate list of x_i, early exit, binary64 recheck), but the
// denominators den_rc = u_r . w_c of a tile of 128 rays against 32 candidates
// come from one `tcgen05.mma.kind::f16` (A = ray directions [128 x 16],
// B = candidate offsets [32 x 16], fp16 operands with d padded to K = 16,
// fp32 accumulation in tensor memory).  Each thread owns one ray (one
// tensor-memory lane), reads its 32 den values with `tcgen05.ld` and runs the
// interval screening with an error bound that covers the fp16 rounding of
// both operands and the tensor-core accumulation.
//
#include <algorithm>
#include <cmath>

#include "vd_mc_common.cuh"
#include "vd_tc.cuh"

namespace vd {

namespace {

constexpr int kTcThreads = 128;  // rays per tile = MMA M = tensor-memory lanes
constexpr int kTcN = 32;         // candidates per MMA (MMA N, tensor-memory columns)
constexpr int kTcBuf = 8;        // candidates kept per ray

__host__ __device__ inline size_t tc_smem(int K) {
  const size_t Kp = ((size_t)K + kTcN - 1) / kTcN * kTcN;
  return Kp * 32 + (size_t)kTcThreads * 32 + Kp * 5 * 4 + (size_t)kTcThreads * kTcBuf * 8 +
         (size_t)kTcThreads * (kTcN + 1) * 4;
}


template <int D>
__global__ void __launch_bounds__(kTcThreads) k_mc_cell_tc(TreeView tr, int64_t R, uint64_t seed, uint32_t set,
                                                           RayOut ro, Counters* ctr, unsigned long long* work,
                                                           int32_t* fb_cell, int32_t* fb_ray, int64_t fb_cap,
                                                           long long wait_limit) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int64_t s_cell;
  const int K = tr.K;
  const int Kp = (K + kTcN - 1) / kTcN * kTcN;
  unsigned char* B16 = smem;                          // [Kp x 16] fp16 candidate offsets
  unsigned char* A16 = smem + (size_t)Kp * 32;        // [128 x 16] fp16 ray directions
  float* snlo = reinterpret_cast<float*>(A16 + kTcThreads * 32);
  float* snhi = snlo + Kp;
  float* swn = snhi + Kp;
  float* sflo = swn + Kp;
  int32_t* sid = reinterpret_cast<int32_t*>(sflo + Kp);
  int32_t* cb = reinterpret_cast<int32_t*>(sid + Kp) + threadIdx.x * kTcBuf;
  float* ct = reinterpret_cast<float*>(reinterpret_cast<int32_t*>(sid + Kp) + kTcThreads * kTcBuf) +
              threadIdx.x * kTcBuf;
  // this thread's den row of the current chunk (stride kTcN + 1: no bank conflicts)
  float* sden = reinterpret_cast<float*>(reinterpret_cast<int32_t*>(sid + Kp) + 2 * kTcThreads * kTcBuf) +
                threadIdx.x * (kTcN + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int d = tr.d;
  const float B = tr.coord_abs;
  const float gam = (float)(D + 1) * kU32 * 1.01f;
  const float EW = 4.01f * kU32 * B;
  const float e1 = 1.1f * (gam + 2.1f * kU32);  // |ww32 - |w|^2| <= e1 ww32
  const TcBound eb = tc_bound(D);
  const float a1 = eb.a1, a0 = eb.a0;
  const uint32_t idesc = tc::idesc_f16_f32(kTcThreads, kTcN);

  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, kTcN);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16);
  uint32_t phase = 0;
  bool timed_out = false;
  unsigned long long n_pairs = 0, n_rech = 0;
  const uint64_t adesc = tc::smem_desc(A16, tc::kLbo16, tc::kSbo16);

  while (!timed_out) {
    if (tid == 0) s_cell = (int64_t)atomicAdd(work, 1ull);
    __syncthreads();
    const int64_t i = s_cell;
    __syncthreads();
    if (i >= tr.N) break;
    const int n = tr.kcnt[i];
    const int np = (n + kTcN - 1) / kTcN * kTcN;
    double g64[D];
    float g32[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      g64[k] = k < d ? tr.X[i * d + k] : 0.0;
      g32[k] = k < d ? tr.X32[i * d + k] : 0.f;
    }
    // ---- stage the cell's candidate list: fp16 offsets + binary32 bounds ----
    for (int c = tid; c < np; c += kTcThreads) {
      float h[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) h[k] = 0.f;
      if (c < n) {
        const int32_t id = tr.knn[i * K + c];
        float ww = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float w = k < d ? __double2float_rn(tr.X[(int64_t)id * d + k] - g64[k]) : 0.f;
          ww = fmaf(w, w, ww);
          if (k < 16) h[k] = w;
        }
        snlo[c] = ww * (1.f - e1);
        snhi[c] = ww * (1.f + e1);
        swn[c] = sqrtf(ww) * (1.f + gam);
        sflo[c] = true_d2_lower(ww32_of<D>(tr.X32 + (int64_t)id * d, 1, g32, d), gam, EW, D);
        sid[c] = id;
      }
      tc::store_row16(B16, c, h);
    }
    const float cert_lo = true_d2_lower(tr.kcert[i], gam, EW, D);
    // ---- rays, 128 per tile ----
    for (int64_t t0 = 0; t0 < R; t0 += kTcThreads) {
      const int64_t k = t0 + tid;
      const bool valid = k < R;
      double u64[D];
      float u32[D], p0[D];
      float T = INFINITY;
      int nc = 0;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        u64[q] = 0.0;
        p0[q] = 0.f;
      }
      if (valid) {
        mc_direction<D>(seed, set, (uint32_t)i, (uint32_t)k, d, u64);
        if (ro.u) {
#pragma unroll
          for (int q = 0; q < D; ++q)
            if (q < d) ro.u[(i * R + k) * d + q] = u64[q];
        }
      }
      float hu[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) hu[q] = 0.f;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        u32[q] = __double2float_rn(u64[q]);
        if (q < 16) hu[q] = u32[q];
      }
      tc::store_row16(A16, tid, hu);
      bool overflow = false;
      if (valid) T = mc_faces<D>(u64, u32, g32, d, cb, ct, nc, kTcBuf, overflow);
      Ball<D> ball;
      make_ball<D>(g32, p0, u32, T, B, ball);
      float far2 = far_radius2<D>(tr, ball, g32);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      bool certified = !valid;
      int done = 0;  // candidates screened by this ray
      for (int c0 = 0; c0 < np; c0 += kTcN) {
        if (tid == 0) {
          tc::fence_after_sync();
          tc::mma_f16(tbase, adesc, tc::smem_desc(B16 + (size_t)c0 * 32, tc::kLbo16, tc::kSbo16), idesc, 0u);
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
          float den[kTcN];
          tc::tmem_ld32(taddr, den);
#pragma unroll
          for (int j = 0; j < kTcN; ++j) sden[j] = den[j];
        }
        if (!certified) {
          const int jn = min(kTcN, n - c0);
#pragma unroll 1
          for (int j = 0; j < jn; ++j) {
            const int c = c0 + j;
            if (sflo[c] >= far2) {
              certified = true;
              break;
            }
            done = c + 1;
            const float e = fmaf(a1, swn[c], a0);
            const float dj = sden[j];
            const float dh = dj + e;
            const float nlo = snlo[c];
            if (!(dh > 0.f) || nlo > 2.f * T * dh * (1.f + 8.f * kU32)) continue;
            const float dl = dj - e;
            const float thi = dl > 0.f ? __fdiv_rn(snhi[c], 2.f * dl) * (1.f + 4.f * kU32) : INFINITY;
            const float tlo = __fdiv_rn(nlo, 2.f * dh) * (1.f - 4.f * kU32);
            if (thi < T) {
              T = thi;
              make_ball<D>(g32, p0, u32, T, B, ball);
              far2 = far_radius2<D>(tr, ball, g32);
            }
            if (!overflow) overflow = !mc_push(sid[c], tlo, T, cb, ct, nc, kTcBuf);
          }
        }
        const bool more = !certified && (c0 + kTcN < n);
        tc::fence_before_sync();
        if (!__syncthreads_or(more)) break;
      }
      if (timed_out) break;
      if (valid) {
        n_pairs += (unsigned long long)done;
        if (!certified) certified = cert_lo >= far2;
        if (!certified || overflow) {
          const unsigned long long q = atomicAdd(&ctr->fallback, 1ull);
          if ((int64_t)q < fb_cap) {
            fb_cell[q] = (int32_t)i;
            fb_ray[q] = (int32_t)k;
          } else {
            atomicOr(&ctr->flags, kFlagQueue);
          }
          ro.t[i * R + k] = (double)T;  // the bound found so far seeds the tree walk
        } else {
          mc_recheck<D>(tr.X, d, g64, u64, cb, ct, nc, T, ro.hit[i * R + k], ro.t[i * R + k], n_rech);
        }
      }
      __syncthreads();  // the next tile rewrites the A operand
    }
    __syncthreads();  // the next cell rewrites the B operand
  }
  if (timed_out) {
    // give the in-flight MMA a bounded chance to finish before freeing its memory
    // the MMA still in flight must finish before its tensor memory is freed:
    // this wait has its own generous bound, whatever limit gave up above
    tc::mbar_wait(&mbar, phase ^ 1u, wait_limit > (1ll << 24) ? wait_limit : (1ll << 24));
    if (tid == 0) atomicOr(&ctr->flags, kFlagTimeout);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, kTcN);
  for (int o = 16; o; o >>= 1) {
    n_pairs += __shfl_xor_sync(kFull, n_pairs, o);
    n_rech += __shfl_xor_sync(kFull, n_rech, o);
  }
  if ((tid & 31) == 0) {
    atomicAdd(&ctr->pairs, n_pairs);
    atomicAdd(&ctr->rechecked, n_rech);
  }
}

template <int D>
cudaError_t launch_tc_d(const TreeView& tv, int64_t R, uint64_t seed, uint32_t set, const RayOut& ro, Counters* ctr,
                        unsigned long long* work, int32_t* fb_cell, int32_t* fb_ray, int64_t fb_cap,
                        long long wait_limit, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t sm = tc_smem(tv.K);
  allow_max_dyn_smem(k_mc_cell_tc<D>);
  // The occupancy API reports one block per SM for any kernel that allocates
  // tensor memory; the resident count follows from registers, shared memory
  // and warps, and 16 blocks of 32 columns fill the 512 tensor-memory columns.
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, k_mc_cell_tc<D>);
  int smem_sm = 0, regs_sm = 0, warps_sm = 0;
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&warps_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  const int warps = kTcThreads / 32;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  const int by_regs = regs_sm / std::max(1, regs_warp * warps);
  const int by_smem = (int)(smem_sm / (sm + fa.sharedSizeBytes + 1024));
  const int by_warps = warps_sm / 32 / warps;
  const int occ = std::max(1, std::min(std::min(by_regs, by_smem), std::min(by_warps, 16)));
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * occ, tv.N));
  cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
  k_mc_cell_tc<D><<<(unsigned)grid, kTcThreads, sm, st>>>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap,
                                                           wait_polls(wait_limit));
  count_launch();
  return cudaGetLastError();
}

}  // namespace

// Tensor-core variant of launch_mc_cells (same contract).
cudaError_t launch_mc_cells_tc(const TreeView& tv, int64_t R, uint64_t seed, uint32_t set, const RayOut& ro,
                               Counters* ctr, long long wait_limit, cudaStream_t st, int64_t* nfallback) {
  unsigned long long* work = reinterpret_cast<unsigned long long*>(&ctr->aux1);
  int32_t* fb_cell = ro.fallback_list;
  int32_t* fb_ray = ro.fallback_list + ro.fallback_cap / 2;
  const int64_t fb_cap = ro.fallback_cap / 2;
  cudaMemsetAsync(&ctr->fallback, 0, sizeof(unsigned long long), st);
  cudaError_t e;
  switch (tv.d) {
    case 1: e = launch_tc_d<1>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wait_limit, st); break;
    case 2: e = launch_tc_d<2>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wait_limit, st); break;
    case 3: e = launch_tc_d<3>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wait_limit, st); break;
    case 4: e = launch_tc_d<4>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wait_limit, st); break;
    case 5: e = launch_tc_d<5>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wait_limit, st); break;
    case 6: e = launch_tc_d<6>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wait_limit, st); break;
    case 7:
    case 8: e = launch_tc_d<8>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wait_limit, st); break;
    case 9: case 10: case 11: case 12:
      e = launch_tc_d<12>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wait_limit, st);
      break;
    default: e = launch_tc_d<16>(tv, R, seed, set, ro, ctr, work, fb_cell, fb_ray, fb_cap, wait_limit, st); break;
  }
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
