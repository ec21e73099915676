// vd_ray_tc.cu -- the candidate-list RayCast of explicit rays (vertex
// traversal, random walks, vd_raycast) with its screening contraction on the
// tensor cores (Section 2.2, Eq. (t), Algorithm 1).
//
// For a ray from v along u with reference generator g, node j beats the bound
// T exactly when f_j = |w_j|^2 - 2 p.w_j - 2 T u.w_j <= 0 with w_j = x_j - g,
// p = v - g (the incircle criterion of Section 2.2 written with Eq. (t)'s
// numerator and denominator).  Rays of one traversal level that share g scan
// the same sorted candidate list of g, so the rays are grouped by g (a
// counting sort per call) and a block takes one group at a time:
//
//   * A = 128 consecutive list entries w_j (fp16, d padded to K = 16),
//     B = the group's rays, two rows each: u_i and p_i (fp16);
//   * one `tcgen05.mma.kind::f16` (M = 128, N = 2 x rays, K = 16, fp32
//     accumulation) puts u_i.w_j and p_i.w_j in tensor memory, lane j =
//     entry j, so each thread owns one list entry and reads its row with
//     `tcgen05.ld`;
//   * pass A (first chunk only): per (ray, entry) an upper bound of t_j from
//     the tensor-core values with a proven error margin; the block minimum
//     per ray tightens the ray's bound T_i;
//   * pass B: the test f_j <= margin with T_i; the few pairs that pass it
//     are screened again in binary32 exactly as the one-thread list scan
//     does, and kept as candidates when their lower bound of t_j does not
//     exceed T_i;
//   * a ray is done once the last entry of a chunk lies beyond the reach of
//     its ball (the list is sorted by distance from g), and the binary64
//     recheck of its candidates decides the hit in the canonical order.
//
// The per-ray binary64 steps run on full warps in kernels of their own: the
// scatter of the counting sort also writes each ray's record (binary32
// copies of the ray, norms for the error bounds, the box-face bound) before
// the tensor-core kernel, which only screens, and a finish kernel (binary64
// recheck of the node candidates and of the faces) runs after it.
//
// Error of one tensor-core dot product of binary32 vectors a, w rounded to
// fp16 with fp32 accumulation: 2^-11 relative per operand component (2^-25
// absolute below the fp16 normal range) and 2^-16 of the sum of |products|
// for the accumulation, i.e. at most (2^-10 + 2^-15 + 2^-22)|a||w| +
// 2^-25 sqrt(d)(|a| + |w|) + d 2^-50.  The binary32 inputs differ from the
// exact ones by the bounds the binary32 screening already uses.
#include <algorithm>
#include <climits>
#include <cmath>

#include "vd_internal.h"
#include "vd_ray_common.cuh"
#include "vd_tc.cuh"

namespace vd {

namespace {

constexpr int kGrpRays = 32;            // rays per work item
constexpr int kGrpCols = 2 * kGrpRays;  // MMA N at most = tensor-memory columns
constexpr int kGrpM = 128;              // list entries per chunk = MMA M = threads
constexpr int kGrpCand = 16;            // node candidates kept per ray (more: binary64 path)

// Per-ray records in grouped order (slot s = position in perm), 32-bit words.
// In (prep -> tensor-core kernel): u32[D] p32[D] eta[D+1] U1 P1 P2 U2 hasp
// Tface m, padded to a multiple of 4.  Out (tensor-core kernel -> finish):
// T state nc - | (cid, ctlo) x kGrpCand, the pairs interleaved so that the
// header and the first two candidates share one 32-byte sector.
template <int D>
struct Rin {
  static constexpr int U = 0, P = D, ETA = 2 * D, U1 = 3 * D + 1, P1 = U1 + 1, P2 = U1 + 2, U2 = U1 + 3,
                       HASP = U1 + 4, T = U1 + 5, M = U1 + 6;
  static constexpr int W = (3 * D + 8 + 3) / 4 * 4;
};
constexpr int kRinMax = 32;
static_assert(Rin<8>::W == kRinMax, "the largest prep record");
constexpr int kRout = 4 + 2 * kGrpCand;
enum : int { kOutT = 0, kOutState, kOutNc, kOutCand = 4 };

// Scratch of one call, carved from RayOut::grp_buf (int32 units):
// cnt[N] fill[N] tot[4] | start[N] | perm[R] | pad | items[R/32 + N + 1]
// (int4) | rin[R][<= kRinMax] | rout[R][kRout].
struct GrpLayout {
  int32_t* cnt;    // rays per reference node
  int32_t* fill;   // rays placed so far per node
  uint32_t* tot;   // [0] work items, [1] rays
  int32_t* start;  // first slot of each node's rays in perm
  int32_t* perm;   // ray indices grouped by reference node
  int4* items;     // (g, first slot, rays) per work item
  int64_t item_cap;
  float* rin;      // per slot, Rin<D>::W words
  float* rout;     // per slot, kRout words
};

GrpLayout grp_layout(int32_t* buf, int64_t N, int64_t R) {
  GrpLayout L;
  L.cnt = buf;
  L.fill = buf + N;
  L.tot = reinterpret_cast<uint32_t*>(buf + 2 * N);
  L.start = buf + 2 * N + 4;
  L.perm = L.start + N;
  const int64_t off = (3 * N + 4 + R + 3) / 4 * 4;  // 16-byte aligned
  L.items = reinterpret_cast<int4*>(buf + off);
  L.item_cap = R / kGrpRays + N + 1;
  const int64_t off2 = off + 4 * L.item_cap;
  L.rin = reinterpret_cast<float*>(buf + off2);
  L.rout = reinterpret_cast<float*>(buf + off2 + (int64_t)kRinMax * R);
  return L;
}

__device__ __forceinline__ int32_t ref_node(const RaySource& rs, int64_t r, int64_t N) {
  const int32_t g = rs.eta[r * rs.eta_stride];
  return (g < 0 || g >= N) ? 0 : g;  // a bad reference is flagged by the prep kernel
}

__device__ __forceinline__ int64_t ray_count(const RaySource& rs) {
  return rs.R_dev ? min((int64_t)*rs.R_dev, rs.R) : rs.R;
}

__global__ void k_grp_count(RaySource rs, int64_t N, int32_t* cnt) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < ray_count(rs)) atomicAdd(&cnt[ref_node(rs, r, N)], 1);
}

// One thread per node: the node's rays get a contiguous range of perm and
// ceil(count / kGrpRays) work items (warp-aggregated atomics).
__global__ void k_grp_alloc(const int32_t* cnt, int64_t N, int32_t* start, int4* items, int64_t item_cap,
                            uint32_t* tot, unsigned* flags) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int c = g < N ? cnt[g] : 0;
  const int nit = (c + kGrpRays - 1) / kGrpRays;
  int sc = c, si = nit;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, sc, o), z = __shfl_up_sync(kFull, si, o);
    if (lane >= o) {
      sc += y;
      si += z;
    }
  }
  uint32_t bc = 0, bi = 0;
  if (lane == 31) {
    bc = atomicAdd(&tot[1], (uint32_t)sc);
    bi = atomicAdd(&tot[0], (uint32_t)si);
  }
  bc = __shfl_sync(kFull, bc, 31);
  bi = __shfl_sync(kFull, bi, 31);
  if (c == 0) return;
  const int base = (int)bc + sc - c;
  const int64_t ib = (int64_t)bi + si - nit;
  start[g] = base;
  for (int q = 0; q < nit; ++q) {
    if (ib + q < item_cap) items[ib + q] = make_int4((int)g, base + q * kGrpRays, min(kGrpRays, c - q * kGrpRays), 0);
    else atomicOr(flags, kFlagQueue);
  }
}

// Order-preserving map of binary32 values to int (for atomicMin on a bound).
__device__ __forceinline__ int fkey(float x) {
  const int i = __float_as_int(x);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float fval(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// Binary32 interval [tlo, thi] of the box face of axis a the ray leaves
// through, t = (b - v_a) / u_a (face_bounds32); false if u_a = 0 or the face
// is in eta.
template <int D>
__device__ __forceinline__ bool face_interval(const double (&v)[D], const double (&u)[D], const float (&u32)[D],
                                              const int32_t (&eta)[D + 1], int m, int a, int32_t& fid, float& tlo,
                                              float& thi) {
  float ua = 0.f;
  double ua64 = 0.0, va64 = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (k == a) {
      ua = u32[k];
      ua64 = u[k];
      va64 = v[k];
    }
  const int sd = face_bounds32(ua, ua64, __double2float_rn(va64), tlo, thi);
  if (sd < 0) return false;
  fid = face_id(a, sd);
  for (int q = 0; q < m; ++q)
    if (eta[q] == fid) return false;
  return true;
}

// Loads ray r and its binary32 copies (reference node g = eta[0]); a bad
// reference is flagged and replaced by node 0, as the other kernels do.
template <int D>
__device__ __forceinline__ void grp_load_ray(const TreeView& tr, const RaySource& rs, Counters* ctr, int64_t r,
                                             double (&v)[D], double (&u)[D], int32_t (&eta)[D + 1], int& m,
                                             float (&u32)[D]) {
  load_ray<D>(tr, rs, r, v, u, eta, m);
  if (m < 1 || eta[0] < 0 || eta[0] >= tr.N) {
    atomicOr(&ctr->flags, kFlagBadInput);
    m = 1;
    eta[0] = 0;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) u32[k] = __double2float_rn(u[k]);
}

// Scatter and prep, one thread per ray (full warps): the ray takes the next
// slot of its reference node's range of perm, and its record holds the
// binary32 direction and offset p = v - g, the norms the error bounds need
// and the face bound.
template <int D>
__global__ void k_grp_scatter(TreeView tr, RaySource rs, Counters* ctr, GrpLayout L) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= ray_count(rs)) return;
  const int d = tr.d;
  const int32_t gref = ref_node(rs, r, tr.N);
  const int64_t s = L.start[gref] + atomicAdd(&L.fill[gref], 1);
  L.perm[s] = (int32_t)r;
  double v[D], u[D];
  int32_t eta[D + 1];
  int m;
  float u32[D];
  grp_load_ray<D>(tr, rs, ctr, r, v, u, eta, m, u32);
  const int32_t g = eta[0];
  using I = Rin<D>;
  float rec[I::W];
#pragma unroll
  for (int k = 0; k < I::W; ++k) rec[k] = 0.f;
  float U1 = 0.f, U2s = 0.f, P1 = 0.f, P2s = 0.f;
  bool hasp = false;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double gk = k < d ? tr.X[(int64_t)g * d + k] : 0.0;
    const double pk = __dadd_rn(v[k], -gk);
    rec[I::U + k] = u32[k];
    rec[I::P + k] = __double2float_rn(pk);
    U1 += fabsf(u32[k]);
    U2s = fmaf(u32[k], u32[k], U2s);
    const float pa = fabsf(__double2float_ru(fabs(pk)));
    P1 += pa;
    P2s = fmaf(pa, pa, P2s);
    hasp |= (pk != 0.0);
  }
  float T = INFINITY;
  if (rs.box)
    for (int a = 0; a < d; ++a) {
      int32_t fid;
      float tlo, thi;
      if (face_interval<D>(v, u, u32, eta, m, a, fid, tlo, thi)) T = fminf(T, thi);
    }
  rec[I::U1] = U1 * 1.0001f;
  rec[I::P1] = P1 * 1.0001f;
  rec[I::P2] = sqrtf(P2s) * 1.0001f;
  rec[I::U2] = sqrtf(U2s);  // the kernel adds its rounding margin
  rec[I::HASP] = hasp ? 1.f : 0.f;
  rec[I::T] = T;
  rec[I::M] = __int_as_float(m);
#pragma unroll
  for (int q = 0; q <= D; ++q) rec[I::ETA + q] = __int_as_float(q < m ? eta[q] : kNoId);
  float4* dst = reinterpret_cast<float4*>(L.rin + s * I::W);
#pragma unroll
  for (int k = 0; k < I::W / 4; ++k) dst[k] = make_float4(rec[4 * k], rec[4 * k + 1], rec[4 * k + 2], rec[4 * k + 3]);
}

// Per-ray state of a work item, in shared memory.
template <int D>
struct GrpRay {
  float u[kGrpRays][D];    // binary32 direction
  float p[kGrpRays][D];    // binary32 p = v - g
  // a0 a1 b0c b2 | m1d m0d m1p m0p | bA cA U2 P2 | beta gamma0 Tsnap hasp
  float k[kGrpRays][16];
  int T[kGrpRays];         // running bound (fkey)
  int32_t eta[kGrpRays][D + 1];
  int m[kGrpRays];
  int nc[kGrpRays];
  int32_t cid[kGrpRays][kGrpCand];
  float ctlo[kGrpRays][kGrpCand];
  int state[kGrpRays];     // bit 0 done, bit 1 certified, bit 2 candidate overflow
};
enum : int { kStDone = 1, kStCert = 2, kStOver = 4, kStAbandoned = 8 };

// Ray slot i of a work item belongs to thread (i mod 4) * 32 + i / 4, so the
// per-ray steps (load, exit test, store) of a group spread over the four
// warps.
__device__ __forceinline__ int slot_of_thread(int t) { return (t & 31) < kGrpRays / 4 ? ((t & 31) << 2) | (t >> 5) : -1; }

struct GrpConst {
  float gam, EW, B, sD, c1, ctiny, alpha;
};

// Ray slot i from its prep record: binary32 vectors, the screening
// constants, the tensor-core error terms, the face bound; B operand rows 2i
// (u) and 2i + 1 (p).
template <int D>
__device__ __forceinline__ void grp_ray_load(const float* rec, const GrpConst& C, GrpRay<D>& S, unsigned char* sB,
                                             int i) {
  using I = Rin<D>;
  float r[I::W];
  const float4* src = reinterpret_cast<const float4*>(rec);
#pragma unroll
  for (int k = 0; k < I::W / 4; ++k) {
    const float4 f = src[k];
    r[4 * k] = f.x;
    r[4 * k + 1] = f.y;
    r[4 * k + 2] = f.z;
    r[4 * k + 3] = f.w;
  }
  float hu[16], hp[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    hu[k] = k < D ? r[I::U + k] : 0.f;
    hp[k] = k < D ? r[I::P + k] : 0.f;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    S.u[i][k] = r[I::U + k];
    S.p[i][k] = r[I::P + k];
  }
  const float U1 = r[I::U1], P1 = r[I::P1], P2 = r[I::P2];
  const float U2 = r[I::U2] * (1.f + 2.f * C.gam) + 1e-30f;
  // binary32 screening constants (as the one-thread list scan), then the
  // tensor-core errors |u.w - den_tc| <= m1d |w| + m0d and
  // |p.w - pw_tc| <= m1p |w| + m0p, and pass A's |num| margin terms
  float* K = S.k[i];
  K[0] = 1.1f * C.EW * U1;                                                       // a0
  K[1] = 1.1f * (C.gam + kU32);                                                  // a1
  K[2] = 1.1f * ((float)D * C.EW * C.EW + 2.f * C.EW * P1);                      // b0c
  K[3] = 1.1f * (2.f * sqrtf((float)D) * C.EW + 2.f * (C.gam + kU32) * P2);      // b2
  K[4] = C.c1 * U2 + C.ctiny;                                                    // m1d
  K[5] = 1.1f * C.sD * C.EW * U2 + C.ctiny * U2 + 1e-30f;                        // m0d
  K[6] = C.c1 * P2 + C.ctiny;                                                    // m1p
  K[7] = 1.1f * C.sD * C.EW * P2 + C.ctiny * P2 + 1e-30f;                        // m0p
  K[8] = 1.05f * (2.f * C.sD * C.EW + 2.f * K[6]);                               // bA
  K[9] = 1.05f * ((float)D * C.EW * C.EW + 2.f * K[7]) + 1e-30f;                 // cA
  K[10] = U2;
  K[11] = P2;
  K[15] = r[I::HASP];
  const int m = __float_as_int(r[I::M]);
#pragma unroll
  for (int q = 0; q <= D; ++q) S.eta[i][q] = __float_as_int(r[I::ETA + q]);
  S.m[i] = m;
  S.T[i] = fkey(r[I::T]);
  S.nc[i] = 0;
  S.state[i] = 0;
  tc::store_row16(sB, 2 * i, hu);
  tc::store_row16(sB, 2 * i + 1, hp);
}

// Exit test of ray slot i after a chunk whose last entry has the binary32
// squared distance wwlast from g (the list is sorted by it).
template <int D>
__device__ void grp_ray_exit(const TreeView& tr, const GrpConst& C, GrpRay<D>& S, const float (&g32)[D], int i,
                             int32_t g, bool have_last, float wwlast, bool list_end) {
  if (S.state[i] & kStDone) return;
  const float T = fval(S.T[i]);
  float u32[D], p32[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    u32[k] = S.u[i][k];
    p32[k] = S.p[i][k];
  }
  Ball<D> ball;
  make_ball<D>(g32, p32, u32, T, C.B, ball);
  const float far2 = far_radius2<D>(tr, ball, g32);
  int st = S.state[i];
  if (have_last && wwlast >= ww_exit(far2, C.gam, C.EW, D)) {
    st |= kStDone | kStCert;  // this and every later entry lie outside the ball
  } else if (list_end) {
    st |= kStDone;
    if (true_d2_lower(tr.kcert[g], C.gam, C.EW, D) >= far2) st |= kStCert;
  }
  S.state[i] = st;
}

// The record the finish kernel reads: final bound, state, node candidates
// (only the 16-byte groups in use are written).
template <int D>
__device__ __forceinline__ void grp_ray_store(const GrpRay<D>& S, int i, float* rec) {
  const int nc = min(S.nc[i], kGrpCand);
  float4* dst = reinterpret_cast<float4*>(rec);
  dst[0] = make_float4(fval(S.T[i]), __int_as_float(S.state[i]), __int_as_float(nc), 0.f);
  for (int q = 0; q < nc; q += 2) {
    const bool two = q + 1 < nc;
    dst[1 + q / 2] = make_float4(__int_as_float(S.cid[i][q]), S.ctlo[i][q],
                                 __int_as_float(two ? S.cid[i][q + 1] : kNoId), two ? S.ctlo[i][q + 1] : INFINITY);
  }
}

// Blocks per SM: 8 (the 512 tensor-memory columns hold 8 blocks of 64; 64
// registers per thread) for d <= 5, 7 above, where 64 registers would spill.
template <int D>
__global__ void __launch_bounds__(kGrpM, D <= 5 ? 8 : 7)
    k_ray_list_tc(TreeView tr, RaySource rs, RayOut ro, Counters* ctr, GrpLayout L, unsigned long long* work,
                  long long wait_limit) {
  __shared__ __align__(1024) unsigned char sA[kGrpM * 32];     // [128 x 16] fp16 list entries w_j
  __shared__ __align__(1024) unsigned char sB[kGrpCols * 32];  // [64 x 16] fp16: row 2i = u_i, 2i + 1 = p_i
  __shared__ __align__(16) GrpRay<D> S;
  __shared__ float s_wwlast;
  __shared__ int4 s_item[2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = tr.d;
  GrpConst C;
  C.B = tr.coord_abs;
  C.gam = (float)(D + 1) * kU32 * 1.01f;
  C.EW = 4.01f * kU32 * C.B;
  C.sD = sqrtf((float)D) * 1.0001f;
  C.c1 = 1.1f * (0x1p-10f + 0x1p-15f + 0x1p-22f + kU32);  // relative error of one MMA dot product
  C.ctiny = 1.1f * C.sD * 0x1p-25f;                        // fp16 rounding below its normal range
  C.alpha = 1.1f * C.gam + 2.f * kU32;                     // |w|^2 terms of the margins
  const int64_t nitems = min((int64_t)L.tot[0], L.item_cap);
  const int slot = slot_of_thread(tid);

  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, kGrpCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    const unsigned long long w = atomicAdd(work, 1ull);
    s_item[0] = (int64_t)w < nitems ? L.items[w] : make_int4(-1, 0, 0, 0);
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16);
  const uint64_t adesc = tc::smem_desc(sA, tc::kLbo16, tc::kSbo16);
  const uint64_t bdesc = tc::smem_desc(sB, tc::kLbo16, tc::kSbo16);
  uint32_t phase = 0;
  bool timed_out = false;
  unsigned long long n_pairs = 0;

  int it = 0;
  for (; !timed_out; ++it) {
    const int4 item = s_item[it & 1];
    if (item.x < 0) break;
    if (tid == 0) {  // the next item is fetched while this one runs
      const unsigned long long w = atomicAdd(work, 1ull);
      s_item[(it + 1) & 1] = (int64_t)w < nitems ? L.items[w] : make_int4(-1, 0, 0, 0);
    }
    const int32_t g = item.x;
    const int G = item.z;
    const int Gp = (G + 7) & ~7;  // MMA N = 2 Gp, a multiple of 16
    const int n = tr.kcnt[g];
    const int32_t* lst = tr.knn + (int64_t)g * tr.K;
    const uint32_t idesc = tc::idesc_f16_f32(kGrpM, 2 * Gp);
    float g32[D];
#pragma unroll
    for (int k = 0; k < D; ++k) g32[k] = k < d ? tr.X32[(int64_t)g * d + k] : 0.f;

    for (int c0 = 0;; c0 += kGrpM) {
      // ---- stage the chunk: thread j owns list entry c0 + j ----
      const int e = c0 + tid;
      const bool valid = e < n;
      const int32_t id = valid ? lst[e] : kNoId;
      float w[D], ww = 0.f;
      {
        float x[D];
        load_x32<D>(tr, valid ? id : g, valid, x);
        float h[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) h[k] = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          w[k] = (k < d && valid) ? x[k] - g32[k] : 0.f;
          ww = fmaf(w[k], w[k], ww);  // the same expression orders the list
          if (k < 16) h[k] = w[k];
        }
        tc::store_row16(sA, tid, h);
      }
      const float wn = norm_up(ww, C.gam);
      const int last = min(n - c0, kGrpM) - 1;
      if (tid == last) s_wwlast = ww;
      if (c0 == 0 && slot >= 0 && slot < Gp) {  // the item's rays (B operand); padding rows are zero
        if (slot < G) {
          grp_ray_load<D>(L.rin + (int64_t)(item.y + slot) * Rin<D>::W, C, S, sB, slot);
        } else {
          float z[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) z[k] = 0.f;
          tc::store_row16(sB, 2 * slot, z);
          tc::store_row16(sB, 2 * slot + 1, z);
        }
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
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
      n_pairs += valid ? (unsigned long long)G : 0ull;
      // ---- pass A (first chunk): block minimum of the upper bounds of t_j ----
      if (c0 == 0) {
        for (int cb = 0; cb < 2 * Gp; cb += 16) {
          float dv[16];
          tc::tmem_ld16(taddr + (uint32_t)cb, dv);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int i = (cb >> 1) + q;
            if (i >= G) break;  // uniform across the block
            const float den = dv[2 * q], pw = dv[2 * q + 1];
            const float4 md = *reinterpret_cast<const float4*>(&S.k[i][4]);  // m1d m0d m1p m0p
            const float4 ma = *reinterpret_cast<const float4*>(&S.k[i][8]);  // bA cA U2 P2
            const float Ed = fmaf(md.x, wn, md.y);
            const float dl = den - Ed;
            int key = INT_MAX;
            if (valid && dl > 1e-30f) {
              bool ex = false;  // the generators of eta are excluded by id
              for (int qq = 0; qq < S.m[i]; ++qq) ex |= (id == S.eta[i][qq]);
              if (!ex) {
                // num = |w|^2 - 2 p.w within En of fl(ww - 2 pw_tc)
                const float nc_ = fmaf(-2.f, pw, ww);
                const float En = fmaf(C.alpha, ww, fmaf(ma.x, wn, ma.y)) + 2.1f * kU32 * fabsf(nc_);
                const float nh = nc_ + En;
                const float thi = nh >= 0.f ? __fdividef(nh, 2.f * dl) * (1.f + 8.f * kU32)
                                            : __fdividef(nh, 2.f * (den + Ed)) * (1.f - 8.f * kU32);
                key = fkey(thi);
              }
            }
            key = __reduce_min_sync(kFull, key);
            if (lane == 0 && key != INT_MAX) atomicMin(&S.T[i], key);
          }
        }
        __syncthreads();
      }
      // ---- margins of pass B from each ray's current bound ----
      if (slot >= 0 && slot < G) {
        float* K = S.k[slot];
        const float T = fval(S.T[slot]);
        K[12] = 1.05f * (2.f * C.sD * C.EW + 2.f * K[6] + 2.f * T * K[4] + 4.01f * kU32 * (T * K[10] + K[11]));
        K[13] = 1.05f * ((float)D * C.EW * C.EW + 2.f * K[7] + 2.f * T * K[5]) + 1e-30f;
        K[14] = T;
      }
      __syncthreads();
      // ---- pass B: f_j <= margin, then the binary32 interval of t_j ----
      for (int cb = 0; cb < 2 * Gp; cb += 16) {
        float dv[16];
        tc::tmem_ld16(taddr + (uint32_t)cb, dv);  // every lane: the load is warp-collective
        unsigned pm = 0;  // rays of this column block whose ball may hold entry j
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = (cb >> 1) + q;
          if (i >= G) break;
          const float4 mb = *reinterpret_cast<const float4*>(&S.k[i][12]);  // beta gamma0 Tsnap hasp
          const float lhs = fmaf(-2.f, fmaf(mb.z, dv[2 * q], dv[2 * q + 1]), ww);
          const float rhs = fmaf(mb.x, wn, fmaf(C.alpha, ww, mb.y));
          if (valid && (!(mb.z < INFINITY) || lhs <= rhs)) pm |= 1u << q;
        }
        while (pm) {
          const int i = (cb >> 1) + __ffs(pm) - 1;
          pm &= pm - 1u;
          bool okid = true;
          for (int qq = 0; qq < S.m[i]; ++qq) okid &= (id != S.eta[i][qq]);
          if (!okid) continue;
          const float* K = S.k[i];
          float den = 0.f, pw = 0.f;
#pragma unroll
          for (int k = 0; k < D; ++k) den = fmaf(S.u[i][k], w[k], den);
          if (K[15] != 0.f) {
#pragma unroll
            for (int k = 0; k < D; ++k) pw = fmaf(S.p[i][k], w[k], pw);
          }
          const float num = fmaf(-2.f, pw, ww);
          const float Eden = fmaf(K[1], wn, K[0]);
          const float dh = den + Eden;
          if (!(dh > 0.f)) continue;
          const float Enum = fmaf(1.1f * kU32, fabsf(num), fmaf(1.1f * C.gam, ww, fmaf(K[3], wn, K[2])));
          const float nlo = num - Enum;
          const float Tc = fval(S.T[i]);
          if (!(nlo <= 0.f || nlo <= 2.f * Tc * dh * (1.f + 8.f * kU32))) continue;
          const float dl = den - Eden;
          const float nhi = num + Enum;
          float thi = INFINITY, tlo = -INFINITY;
          if (dl > 0.f)
            thi = nhi >= 0.f ? __fdiv_rn(nhi, 2.f * dl) * (1.f + 4.f * kU32)
                             : __fdiv_rn(nhi, 2.f * dh) * (1.f - 4.f * kU32);
          if (nlo > 0.f) tlo = __fdiv_rn(nlo, 2.f * dh) * (1.f - 4.f * kU32);
          if (thi < Tc) atomicMin(&S.T[i], fkey(thi));
          if (tlo <= fminf(Tc, thi)) {
            const int pos = atomicAdd(&S.nc[i], 1);
            if (pos < kGrpCand) {
              S.cid[i][pos] = id;
              S.ctlo[i][pos] = tlo;
            } else {
              atomicOr(&S.state[i], kStOver);
            }
          }
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      // ---- exit: a ray is done once the chunk's last entry is beyond its ball ----
      if (slot >= 0 && slot < G) grp_ray_exit<D>(tr, C, S, g32, slot, g, last >= 0, s_wwlast, c0 + kGrpM >= n);
      if (!__syncthreads_or(slot >= 0 && slot < G && !(S.state[slot] & kStDone))) break;
    }
    if (timed_out) break;
    if (slot >= 0 && slot < G) grp_ray_store<D>(S, slot, L.rout + (int64_t)(item.y + slot) * kRout);
    __syncthreads();  // the next item rewrites the ray state and the B operand
  }
  if (timed_out) {
    // the MMA still in flight must finish before its tensor memory is freed:
    // this wait has its own generous bound, whatever limit gave up above
    tc::mbar_wait(&mbar, phase ^ 1u, wait_limit > (1ll << 24) ? wait_limit : (1ll << 24));
    if (tid == 0) atomicOr(&ctr->flags, kFlagTimeout);
    // every ray of this block's unfinished items, and of the items still
    // queued, is marked abandoned: the finish kernel writes "no hit" for it
    __syncthreads();
    for (int k = 0;; ++k) {
      int4 itm;
      if (k < 2) {
        itm = s_item[(it + k) & 1];
      } else {
        __syncthreads();
        if (tid == 0) {
          const unsigned long long w = atomicAdd(work, 1ull);
          s_item[0] = (int64_t)w < nitems ? L.items[w] : make_int4(-1, 0, 0, 0);
        }
        __syncthreads();
        itm = s_item[0];
      }
      if (itm.x < 0) {
        if (k == 0) continue;  // nothing was current: look at the prefetched item
        if (k >= 1) break;
      }
      for (int q = tid; q < itm.z; q += kGrpM)
        L.rout[(int64_t)(itm.y + q) * kRout + kOutState] = __int_as_float(kStAbandoned);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, kGrpCols);
  for (int o = 16; o; o >>= 1) n_pairs += __shfl_xor_sync(kFull, n_pairs, o);
  if (lane == 0) atomicAdd(&ctr->pairs, n_pairs);
}


// Finish, one thread per slot (full warps): the tree walk for rays the list
// could not certify (with the bound found so far), the binary64 path for
// rays whose candidate buffer overflowed, else the binary64 recheck of the
// node candidates and of the box faces whose lower bound does not exceed T,
// in the canonical order; "no hit" for rays a timed-out kernel abandoned.
template <int D>
__global__ void k_grp_finish(TreeView tr, RaySource rs, RayOut ro, Counters* ctr, GrpLayout L) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int d = tr.d;
  unsigned long long n_rech = 0;
  if (s < ray_count(rs)) {
    const int64_t r = L.perm[s];
    const float* rec = L.rout + s * kRout;
    const float4 h = *reinterpret_cast<const float4*>(rec);  // T state nc -
    const int st = __float_as_int(h.y);
    const float T = h.x;
    const int64_t op = out_pos(rs, ro, r);
    if (st & kStAbandoned) {
      ro.hit[op] = kNoId;
      ro.t[op] = NAN;
    } else if (!(st & kStCert)) {  // finished by the tree walk, from the bound found so far
      const unsigned long long k = atomicAdd(&ctr->fallback, 1ull);
      if ((int64_t)k < ro.fallback_cap) ro.fallback_list[k] = (int32_t)r;
      else atomicOr(&ctr->flags, kFlagQueue);
      ro.t[op] = (double)T;
    } else if (st & kStOver) {  // redone on the binary64 path
      const unsigned long long k = atomicAdd(&ctr->overflow, 1ull);
      if ((int64_t)k < ro.overflow_cap) ro.overflow_list[k] = (int32_t)r;
      else atomicOr(&ctr->flags, kFlagCandOverflow);
      ro.hit[op] = kNoId;
      ro.t[op] = NAN;
    } else {
      double v[D], u[D];
      int32_t eta[D + 1];
      int m;
      float u32[D];
      grp_load_ray<D>(tr, rs, ctr, r, v, u, eta, m, u32);
      const int32_t g = eta[0];
      double bt = INFINITY;
      int bc = 2, bk = 0;
      const int nc = __float_as_int(h.z);
      for (int q = 0; q < nc; ++q) {
        const float2 c = *reinterpret_cast<const float2*>(rec + kOutCand + 2 * q);
        if (!(c.y <= T)) continue;
        const int32_t cid = __float_as_int(c.x);
        ++n_rech;
        double den = 0.0, ww64 = 0.0, pw = 0.0, w64[D];
#pragma unroll
        for (int k = 0; k < D; ++k)
          w64[k] = k < d ? __dadd_rn(tr.X[(int64_t)cid * d + k], -tr.X[(int64_t)g * d + k]) : 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k < d) den = __dadd_rn(den, __dmul_rn(u[k], w64[k]));
        if (!(den > 0.0)) continue;
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k < d) ww64 = __dadd_rn(ww64, __dmul_rn(w64[k], w64[k]));
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k < d) pw = __dadd_rn(pw, __dmul_rn(__dadd_rn(v[k], -tr.X[(int64_t)g * d + k]), w64[k]));
        const double num = __dadd_rn(ww64, -__dmul_rn(2.0, pw));
        const double t = __ddiv_rn(num, __dmul_rn(2.0, den));
        if (better(t, 0, cid, bt, bc, bk)) {
          bt = t;
          bc = 0;
          bk = cid;
        }
      }
      if (rs.box)
        for (int a = 0; a < d; ++a) {
          int32_t fid;
          float tlo, thi;
          if (!face_interval<D>(v, u, u32, eta, m, a, fid, tlo, thi) || !(tlo <= T)) continue;
          ++n_rech;
          const int sd = face_side(fid);
          double ua = 0.0, va = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k)
            if (k == a) {
              ua = u[k];
              va = v[k];
            }
          const double t = __ddiv_rn(__dadd_rn(sd ? 1.0 : 0.0, -va), ua);
          if (better(t, 1, 2 * a + sd, bt, bc, bk)) {
            bt = t;
            bc = 1;
            bk = 2 * a + sd;
          }
        }
      ro.hit[op] = gen_from_key(bc, bk);
      ro.t[op] = bt;
      if (ro.screen_err) ro.screen_err[op] = (bt > 0.0 && bt < INFINITY) ? (float)((T - bt) / bt) : 0.f;
    }
  }
  for (int o = 16; o; o >>= 1) n_rech += __shfl_xor_sync(kFull, n_rech, o);
  if ((threadIdx.x & 31) == 0 && n_rech) atomicAdd(&ctr->rechecked, n_rech);
}

template <int D>
cudaError_t launch_list_tc_d(const TreeView& tv, const RaySource& rs, const RayOut& ro, Counters* ctr,
                             cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t N = tv.N, R = rs.R;
  const GrpLayout L = grp_layout(ro.grp_buf, N, R);
  cudaError_t e = cudaMemsetAsync(L.cnt, 0, (size_t)(2 * N + 4) * sizeof(int32_t), st);  // cnt, fill, tot
  if (e != cudaSuccess) return e;
  const unsigned rb = (unsigned)((R + 255) / 256), nbk = (unsigned)((N + 255) / 256);
  k_grp_count<<<rb, 256, 0, st>>>(rs, N, L.cnt);
  count_launch();
  k_grp_alloc<<<nbk, 256, 0, st>>>(L.cnt, N, L.start, L.items, L.item_cap, L.tot, &ctr->flags);
  count_launch();
  k_grp_scatter<D><<<(unsigned)((R + 127) / 128), 128, 0, st>>>(tv, rs, ctr, L);
  count_launch();
  unsigned long long* work = reinterpret_cast<unsigned long long*>(&ctr->aux1);
  if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
  // The occupancy API reports one block per SM for kernels that allocate
  // tensor memory; registers, shared memory and the 512 tensor-memory
  // columns (8 blocks of 64) set the resident count.
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, k_ray_list_tc<D>);
  int smem_sm = 0, regs_sm = 0;
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  const int regs_blk = (fa.numRegs * 32 + 255) / 256 * 256 * (kGrpM / 32);
  const int by_regs = regs_sm / std::max(1, regs_blk);
  const int by_smem = (int)(smem_sm / (fa.sharedSizeBytes + 1024));
  const int occ = std::max(1, std::min(std::min(by_regs, by_smem), 512 / kGrpCols));
  const long long wl = wait_polls(rs.wait_limit);
  k_ray_list_tc<D><<<(unsigned)((int64_t)nsm * occ), kGrpM, 0, st>>>(tv, rs, ro, ctr, L, work, wl);
  count_launch();
  k_grp_finish<D><<<(unsigned)((R + 127) / 128), 128, 0, st>>>(tv, rs, ro, ctr, L);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int64_t grp_ray_ints(int64_t N, int64_t R) {
  return (3 * N + 4 + R + 3) / 4 * 4 + 4 * (R / kGrpRays + N + 1) + (int64_t)(kRinMax + kRout) * R;
}

cudaError_t launch_list_tc(const TreeView& tv, const RaySource& rs, const RayOut& ro, Counters* ctr,
                           cudaStream_t st) {
  if (rs.R <= 0) return cudaSuccess;
  switch (tv.d) {
    case 1: return launch_list_tc_d<1>(tv, rs, ro, ctr, st);
    case 2: return launch_list_tc_d<2>(tv, rs, ro, ctr, st);
    case 3: return launch_list_tc_d<3>(tv, rs, ro, ctr, st);
    case 4: return launch_list_tc_d<4>(tv, rs, ro, ctr, st);
    case 5: return launch_list_tc_d<5>(tv, rs, ro, ctr, st);
    case 6: return launch_list_tc_d<6>(tv, rs, ro, ctr, st);
    case 7:
    case 8: return launch_list_tc_d<8>(tv, rs, ro, ctr, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vd
