// vd_raycast.cu -- the generic exact RayCast (Section 2.2, Eq. (t),
// Algorithm 1) for arbitrary rays.
//
// Algorithm 1 reaches the first bisector hit by alternating a nearest-
// neighbour query with the projection of Eq. (t); its result is the node
// minimising t_j = (|x_j - v|^2 - |g - v|^2) / (2 u.(x_j - g)) over
// u.(x_j - g) > 0.  This kernel computes that minimum directly: for the
// current bound T, every node with t_j < T lies in the ball centred at
// c = v + T u through g (expand |x_j - c|^2 < |g - c|^2: the difference is
// num_j - 2 T den_j), so a 32-way bounding-box tree is walked nearest box
// first and every box that misses the ball is skipped.
//
// Work layout: a warp owns 32 rays at a time.  Per-ray set-up (binary64
// origin offsets, box faces) runs one ray per lane; the tree walk runs the
// 32 lanes over the 32 nodes of a tile, one ray after the other; the binary64
// recheck again runs one ray per lane, so the binary64 pipe sees full warps.
//
// VD_FP64: every (ray, node) pair is evaluated in binary64 in the canonical
// order and the warp keeps the exact minimum.
// VD_FP32: pairs are screened in binary32 with a rigorous error bound on
// num_j and den_j; a node is kept as candidate when its lower bound on t_j
// does not exceed the running upper bound T, and only the candidates are
// recomputed in binary64 with the canonical formula.
#include <algorithm>
#include <cmath>

#include "vd_dev.cuh"
#include "vd_ray_common.cuh"

namespace vd {

namespace {

constexpr int kWpb = 4;        // warps per block
constexpr int kCmax = 16;      // candidates kept per ray
constexpr int kStk = kFan * kMaxLev;

template <int D>
struct WarpMixed {
  float u[32][D];
  float g[32][D];
  float p[32][D];
  double u64[32][D];
  double p64[32][D];
  float T[32];
  float a0[32], a1[32], b0[32], b2[32];  // per-ray error-bound constants
  int32_t eta[32][D + 1];
  int m[32];
  int hasp[32];
  int ncand[32];
  int32_t cid[32][kCmax];
  float ctlo[32][kCmax];
  int stk[kStk];
};

template <int D>
struct WarpF64 {
  double u[32][D];
  double g[32][D];
  double p[32][D];
  double bt[32];
  int bcls[32], bkey[32];
  int32_t eta[32][D + 1];
  int m[32];
  int stk[kStk];
};

__device__ __forceinline__ int enc(int lev, int64_t idx) { return (lev << 27) | (int)idx; }

template <int D>
__device__ __forceinline__ float box_dist2(const TreeView& tr, int lev, int64_t i, const Ball<D>& b) {
  const int64_t idx = tr.off[lev] + i;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (k < tr.d) {
      const float lo = tr.blo32[k * tr.total + idx], hi = tr.bhi32[k * tr.total + idx];
      const float e = fmaxf(fmaxf(lo - b.c[k], b.c[k] - hi), 0.f);
      s = fmaf(e, e, s);
    }
  }
  return s;
}

// One lane's part of the leaf re-test: lanes k < d add dimension k.
template <int D>
__device__ __forceinline__ bool leaf_alive(const TreeView& tr, int64_t tile, const Ball<D>& b, int lane) {
  float e = 0.f;
  if (lane < tr.d) {
    const int64_t idx = tr.off[0] + tile;
    float ck = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k == lane) ck = b.c[k];
    const float lo = tr.blo32[lane * tr.total + idx], hi = tr.bhi32[lane * tr.total + idx];
    e = fmaxf(fmaxf(lo - ck, ck - hi), 0.f);
    e = e * e;
  }
  return warp_sum(e) * (1.f - 2e-6f) <= b.lim2;
}

// Walks the tree for the ball of the current bound; leaf(tile) evaluates a
// tile and may shrink the ball.
template <int D, class Leaf>
__device__ __forceinline__ void walk(const TreeView& tr, int* stk, Ball<D>& ball, int lane, Leaf&& leaf,
                                     unsigned long long& tiles) {
  int sp = 0;
  if (lane == 0) stk[0] = enc(tr.nlev - 1, 0);
  sp = 1;
  __syncwarp();
  while (sp > 0) {
    const int e = stk[--sp];
    __syncwarp();
    const int lev = e >> 27;
    const int64_t idx = e & ((1 << 27) - 1);
    if (lev == 0) {
      if (leaf_alive<D>(tr, idx, ball, lane)) {
        ++tiles;
        leaf(idx);
      }
      continue;
    }
    const int64_t child = idx * kFan + lane;
    const bool valid = child < tr.cnt[lev - 1];
    float key = INFINITY;  // INFINITY marks "not visited"; a visited child has a finite key
    if (valid) {
      const float d2 = box_dist2<D>(tr, lev - 1, child, ball);
      if (d2 * (1.f - 2e-6f) <= ball.lim2) key = fminf(d2, 3.0e38f);
    }
    int val = (int)child;
    warp_sort(key, val);
    const int n = __popc(__ballot_sync(kFull, key < INFINITY));
    if (lane < n && sp + n - 1 - lane < kStk) stk[sp + n - 1 - lane] = enc(lev - 1, val);
    sp = min(sp + n, kStk);
    __syncwarp();
  }
}

// Same walk for a fixed ball (candidate-list gathering): every box that meets
// the ball is visited, in no particular order, so children are pushed
// without sorting.
template <int D, class Leaf>
__device__ __forceinline__ void walk_fixed(const TreeView& tr, int* stk, const Ball<D>& ball, int lane, Leaf&& leaf) {
  int sp = 0;
  if (lane == 0) stk[0] = enc(tr.nlev - 1, 0);
  sp = 1;
  __syncwarp();
  while (sp > 0) {
    const int e = stk[--sp];
    __syncwarp();
    const int lev = e >> 27;
    const int64_t idx = e & ((1 << 27) - 1);
    if (lev == 0) {  // pushed only if its box meets the ball, which does not change
      leaf(idx);
      continue;
    }
    const int64_t child = idx * kFan + lane;
    const bool in = child < tr.cnt[lev - 1] && box_dist2<D>(tr, lev - 1, child, ball) * (1.f - 2e-6f) <= ball.lim2;
    const unsigned m = __ballot_sync(kFull, in);
    const int pos = sp + __popc(m & ((1u << lane) - 1u));
    if (in && pos < kStk) stk[pos] = enc(lev - 1, child);
    sp = min(sp + __popc(m), kStk);
    __syncwarp();
  }
}

// ------------------------------------------------------------------------
// VD_FP32: binary32 screening + binary64 recheck
// ------------------------------------------------------------------------
template <int D, bool LIST>
__global__ void __launch_bounds__(kWpb * 32) k_ray_mixed(TreeView tr, RaySource rs, RayOut ro, Counters* ctr,
                                                         unsigned long long* work, const int32_t* subset) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpMixed<D>& S = reinterpret_cast<WarpMixed<D>*>(smem_raw)[wib];
  const int d = tr.d;
  const float B = tr.coord_abs;
  const float gam = (float)(D + 1) * kU32 * 1.01f;          // gamma_D for the FMA dot products
  const float EW = 4.01f * kU32 * B;                         // |w32_k - w_k|
  unsigned long long n_tiles = 0, n_pairs = 0, n_rech = 0, n_over = 0;
  int64_t R = rs.R;
  int rpb = rs.rpb;
  if (rs.R_dev) {
    R = min((int64_t)*rs.R_dev, rs.R);
    rpb = R < (int64_t)gridDim.x * kWpb * 64 ? 1 : 32;
  }
  while (true) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(work, 1ull);
    b = __shfl_sync(kFull, b, 0);
    const int64_t b0 = (int64_t)b * rpb;
    if (b0 >= R) break;
    // ---- set-up: one ray per lane ----
    const int64_t slot = b0 + lane;
    const bool vr = lane < rpb && slot < R;
    const int64_t r = vr ? (subset ? (int64_t)subset[slot] : slot) : 0;
    if (vr) {
      double v[D], u[D];
      int32_t eta[D + 1];
      int m;
      load_ray<D>(tr, rs, r, v, u, eta, m);
      if (m < 1 || eta[0] < 0 || eta[0] >= tr.N) {  // g must be a node
        atomicOr(&ctr->flags, kFlagBadInput);
        m = 1;
        eta[0] = 0;
      }
      const int32_t g = eta[0];
      float U1 = 0.f, P1 = 0.f, P2s = 0.f;
      int hasp = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double gk = k < d ? tr.X[(int64_t)g * d + k] : 0.0;
        const double pk = __dadd_rn(v[k], -gk);
        S.u64[lane][k] = u[k];
        S.p64[lane][k] = pk;
        S.u[lane][k] = __double2float_rn(u[k]);
        S.g[lane][k] = __double2float_rn(gk);
        S.p[lane][k] = __double2float_rn(pk);
        U1 += fabsf(S.u[lane][k]);
        const float pa = fabsf(__double2float_ru(fabs(pk)));
        P1 += pa;
        P2s = fmaf(pa, pa, P2s);
        hasp |= (pk != 0.0);
      }
      U1 *= 1.0001f;
      P1 *= 1.0001f;
      const float P2 = sqrtf(P2s) * 1.0001f;
      S.a0[lane] = 1.1f * EW * U1;
      S.a1[lane] = 1.1f * (gam + kU32);
      S.b0[lane] = 1.1f * ((float)D * EW * EW + 2.f * EW * P1);
      S.b2[lane] = 1.1f * (2.f * sqrtf((float)D) * EW + 2.f * (gam + kU32) * P2);
      for (int q = 0; q <= D; ++q) S.eta[lane][q] = q < m ? eta[q] : kNoId;
      S.m[lane] = m;
      S.hasp[lane] = hasp;
      // box faces: binary32 interval of (b - v_a) / u_a
      float T = INFINITY;
      int nc = 0;
      if (rs.box) {
        for (int a = 0; a < d; ++a) {
          float tlo, thi;
          const int s = face_bounds32(S.u[lane][a], u[a], __double2float_rn(v[a]), tlo, thi);
          if (s < 0) continue;
          const int32_t fid = face_id(a, s);
          bool ex = false;
          for (int q = 0; q < m; ++q) ex |= (eta[q] == fid);
          if (ex) continue;
          T = fminf(T, thi);
          if (nc < kCmax) {
            S.cid[lane][nc] = fid;
            S.ctlo[lane][nc] = tlo;
            ++nc;
          }
        }
      }
      if (rs.t_hint) T = fminf(T, (float)ro.t[out_pos(rs, ro, r)]);
      S.T[lane] = T;
      S.ncand[lane] = nc;
    }
    __syncwarp();
    // ---- screening: the warp walks the tree for each ray ----
    for (int rr = 0; rr < rpb && b0 + rr < R; ++rr) {
      float u[D], gg[D], pp[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        u[k] = S.u[rr][k];
        gg[k] = S.g[rr][k];
        pp[k] = S.p[rr][k];
      }
      const float a0 = S.a0[rr], a1 = S.a1[rr], b0c = S.b0[rr], b2 = S.b2[rr];
      const int m = S.m[rr];
      const bool hasp = S.hasp[rr] != 0;
      float T = S.T[rr];
      int nc = S.ncand[rr];
      Ball<D> ball;
      make_ball<D>(gg, pp, u, T, B, ball);
      // screens one node per lane (id, coordinates xs[k * stride]); returns ww32
      auto eval = [&](int32_t id, const float* xs, int stride) -> float {
        bool ok = id != kNoId;
        for (int q = 0; q < m; ++q) ok &= (id != S.eta[rr][q]);
        float w[D];
        float den = 0.f, ww = 0.f, pw = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          w[k] = (k < d) ? xs[k * stride] - gg[k] : 0.f;
          den = fmaf(u[k], w[k], den);
          ww = fmaf(w[k], w[k], ww);
        }
        if (hasp) {
#pragma unroll
          for (int k = 0; k < D; ++k) pw = fmaf(pp[k], w[k], pw);
        }
        const float num = fmaf(-2.f, pw, ww);
        const float wn = sqrtf(ww) * (1.f + gam);
        const float Eden = fmaf(a1, wn, a0);
        const float Enum = fmaf(1.1f * kU32, fabsf(num), fmaf(1.1f * gam, ww, fmaf(b2, wn, b0c)));
        const float dh = den + Eden;
        const float nlo = num - Enum;
        // t_j <= T is possible iff the lower bound of t_j does not exceed T
        const bool cand = ok && dh > 0.f && (nlo <= 0.f || nlo <= 2.f * T * dh * (1.f + 8.f * kU32));
        const unsigned cm = __ballot_sync(kFull, cand);
        if (cm == 0) return ww;
        float thi = INFINITY, tlo = -INFINITY;
        if (cand) {
          const float dl = den - Eden;
          const float nhi = num + Enum;
          if (dl > 0.f)
            thi = nhi >= 0.f ? __fdiv_rn(nhi, 2.f * dl) * (1.f + 4.f * kU32)
                             : __fdiv_rn(nhi, 2.f * dh) * (1.f - 4.f * kU32);
          if (nlo > 0.f) tlo = __fdiv_rn(nlo, 2.f * dh) * (1.f - 4.f * kU32);
        }
        const float Tn = warp_min(thi);
        if (Tn < T) {
          T = Tn;
          make_ball<D>(gg, pp, u, T, B, ball);
        }
        const bool keep = cand && tlo <= T;
        const unsigned km = __ballot_sync(kFull, keep);
        const int nk = __popc(km);
        if (nc >= 0 && nc + nk > kCmax) {
          // compact: drop candidates whose lower bound exceeds the new T
          int cnt = 0;
          for (int c0 = 0; c0 < nc; c0 += 32) {
            const int c = c0 + lane;
            const bool stay = c < nc && S.ctlo[rr][c] <= T;
            const unsigned sm = __ballot_sync(kFull, stay);
            int32_t cidv = 0;
            float ctv = 0.f;
            if (stay) {
              cidv = S.cid[rr][c];
              ctv = S.ctlo[rr][c];
            }
            __syncwarp();
            if (stay) {
              const int pos = cnt + __popc(sm & ((1u << lane) - 1u));
              S.cid[rr][pos] = cidv;
              S.ctlo[rr][pos] = ctv;
            }
            cnt += __popc(sm);
            __syncwarp();
          }
          nc = cnt;
          if (nc + nk > kCmax) nc = -1;  // overflow: the ray is redone on the binary64 path
        }
        if (nc >= 0) {
          if (keep) {
            const int pos = nc + __popc(km & ((1u << lane) - 1u));
            S.cid[rr][pos] = id;
            S.ctlo[rr][pos] = tlo;
          }
          nc += nk;
        }
        __syncwarp();
        return ww;
      };
      if (!LIST) {
        auto leaf = [&](int64_t tile) {
          eval(tr.ids[tile * kTile + lane], tr.x32 + tile * d * kTile + lane, kTile);
        };
        unsigned long long t0 = n_tiles;
        walk<D>(tr, S.stk, ball, lane, leaf, n_tiles);
        n_pairs += (n_tiles - t0) * 32;
      } else {
        // scan g's sorted candidate list; stop once a node is farther from g
        // than 2 rho (it and all later ones lie outside the ball of T)
        const int32_t g = S.eta[rr][0];
        const int32_t* lst = tr.knn + (int64_t)g * tr.K;
        const int n = tr.kcnt[g];
        bool certified = false;
        for (int c0 = 0; c0 < n; c0 += 32) {
          const int c = c0 + lane;
          const int32_t id = c < n ? lst[c] : kNoId;
          const float ww = eval(id, tr.X32 + (int64_t)(c < n ? id : g) * d, 1);
          n_pairs += 32;
          const float far2 = far_radius2<D>(tr, ball, gg);
          const bool far = c < n && true_d2_lower(ww, gam, EW, D) >= far2;
          if (__ballot_sync(kFull, far)) {
            certified = true;
            break;
          }
        }
        if (!certified) certified = true_d2_lower(tr.kcert[g], gam, EW, D) >= far_radius2<D>(tr, ball, gg);
        if (!certified) nc = -2;  // finished by the tree walk
      }
      if (lane == 0) {
        S.T[rr] = T;
        S.ncand[rr] = nc;
      }
      __syncwarp();
    }
    __syncwarp();
    // ---- binary64 recheck: one ray per lane ----
    if (vr) {
      const int nc = S.ncand[lane];
      const int64_t op = out_pos(rs, ro, r);
      if (nc == -2) {
        const unsigned long long k = atomicAdd(&ctr->fallback, 1ull);
        if ((int64_t)k < ro.fallback_cap) ro.fallback_list[k] = (int32_t)r;
        else atomicOr(&ctr->flags, kFlagQueue);
        ro.t[op] = (double)S.T[lane];  // the list's bound seeds the tree walk
      } else if (nc < 0) {
        const unsigned long long k = atomicAdd(&ctr->overflow, 1ull);
        if ((int64_t)k < ro.overflow_cap) ro.overflow_list[k] = (int32_t)r;
        else atomicOr(&ctr->flags, kFlagCandOverflow);
        ++n_over;
        ro.hit[op] = kNoId;
        ro.t[op] = NAN;
      } else {
        const float T = S.T[lane];
        const int32_t g = S.eta[lane][0];
        double bt = INFINITY;
        int bc = 2, bk = 0;
        for (int c = 0; c < nc; ++c) {
          if (!(S.ctlo[lane][c] <= T)) continue;
          const int32_t id = S.cid[lane][c];
          ++n_rech;
          if (id >= 0) {
            double den = 0.0, ww = 0.0, pw = 0.0, w[D];
#pragma unroll
            for (int k = 0; k < D; ++k)
              w[k] = k < d ? __dadd_rn(tr.X[(int64_t)id * d + k], -tr.X[(int64_t)g * d + k]) : 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k)
              if (k < d) den = __dadd_rn(den, __dmul_rn(S.u64[lane][k], w[k]));
            if (!(den > 0.0)) continue;
#pragma unroll
            for (int k = 0; k < D; ++k)
              if (k < d) ww = __dadd_rn(ww, __dmul_rn(w[k], w[k]));
#pragma unroll
            for (int k = 0; k < D; ++k)
              if (k < d) pw = __dadd_rn(pw, __dmul_rn(S.p64[lane][k], w[k]));
            const double num = __dadd_rn(ww, -__dmul_rn(2.0, pw));
            const double t = __ddiv_rn(num, __dmul_rn(2.0, den));
            if (better(t, 0, id, bt, bc, bk)) {
              bt = t;
              bc = 0;
              bk = id;
            }
          } else {
            const int a = face_axis(id), s = face_side(id);
            double va;
            if (rs.mode == 0) va = rs.origins[r * d + a];
            else va = tr.X[(int64_t)g * d + a];
            const double t = __ddiv_rn(__dadd_rn(s ? 1.0 : 0.0, -va), S.u64[lane][a]);
            if (better(t, 1, 2 * a + s, bt, bc, bk)) {
              bt = t;
              bc = 1;
              bk = 2 * a + s;
            }
          }
        }
        ro.hit[op] = gen_from_key(bc, bk);
        ro.t[op] = bt;
        if (ro.screen_err) ro.screen_err[op] = (bt > 0.0 && bt < INFINITY) ? (float)((T - bt) / bt) : 0.f;
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&ctr->tiles, n_tiles);
    atomicAdd(&ctr->pairs, n_pairs);
  }
  for (int o = 16; o; o >>= 1) n_rech += __shfl_xor_sync(kFull, n_rech, o);
  if (lane == 0) atomicAdd(&ctr->rechecked, n_rech);
}

// ------------------------------------------------------------------------
// VD_FP32 over the candidate lists, one thread per ray: each thread scans its
// reference node's sorted list by itself (the warp-per-ray kernel above
// spends warp-wide reductions on every 32 candidates, this one only plain
// per-thread arithmetic), with the same binary32 bounds, the same early exit
// (a candidate whose distance from g exceeds the reach of the current ball
// ends the scan) and the same binary64 recheck.
// ------------------------------------------------------------------------
constexpr int kThrRays = 128;  // threads (rays in flight) per block

// Six blocks per SM at d <= 6 (80 registers): nothing binary64 stays live
// through the scan (the recheck loads the ray again).
template <int D>
__global__ void __launch_bounds__(kThrRays, (D <= 6 ? 6 : D <= 8 ? 4 : 3))
    k_ray_list_thr(TreeView tr, RaySource rs, RayOut ro, Counters* ctr, unsigned long long* work) {
  __shared__ int32_t s_cid[kThrRays][kCmax];
  __shared__ float s_ctlo[kThrRays][kCmax];
  __shared__ int32_t s_eta[kThrRays][D + 1];
  const int tid = threadIdx.x, lane = tid & 31;
  int32_t* cid = s_cid[tid];
  float* ctlo = s_ctlo[tid];
  int32_t* eta = s_eta[tid];
  const int d = tr.d;
  const float B = tr.coord_abs;
  const float gam = (float)(D + 1) * kU32 * 1.01f;
  const float EW = 4.01f * kU32 * B;
  unsigned n_pairs = 0, n_rech = 0;  // per thread; added up in 64 bits at the end
  const int64_t R = rs.R_dev ? min((int64_t)*rs.R_dev, rs.R) : rs.R;
  while (true) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(work, 1ull);
    b = __shfl_sync(kFull, b, 0);
    const int64_t slot = (int64_t)b * 32 + lane;
    if ((int64_t)b * 32 >= R) break;
    if (slot >= R) continue;
    const int64_t r = slot;
    // ---- set-up ----
    double v[D], u[D];
    int m;
    {
      int32_t e[D + 1];
      load_ray<D>(tr, rs, r, v, u, e, m);
      if (m < 1 || e[0] < 0 || e[0] >= tr.N) {
        atomicOr(&ctr->flags, kFlagBadInput);
        m = 1;
        e[0] = 0;
      }
      for (int q = 0; q <= D; ++q) eta[q] = q < m ? e[q] : kNoId;
    }
    const int32_t g = eta[0];
    float u32[D], g32[D], p32[D];
    float U1 = 0.f, P1 = 0.f, P2s = 0.f;
    bool hasp = false;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double gk = k < d ? tr.X[(int64_t)g * d + k] : 0.0;
      const double pk = __dadd_rn(v[k], -gk);
      u32[k] = __double2float_rn(u[k]);
      g32[k] = __double2float_rn(gk);
      p32[k] = __double2float_rn(pk);
      U1 += fabsf(u32[k]);
      const float pa = fabsf(__double2float_ru(fabs(pk)));
      P1 += pa;
      P2s = fmaf(pa, pa, P2s);
      hasp |= (pk != 0.0);
    }
    U1 *= 1.0001f;
    P1 *= 1.0001f;
    const float P2 = sqrtf(P2s) * 1.0001f;
    const float a0 = 1.1f * EW * U1;
    const float a1 = 1.1f * (gam + kU32);
    const float b0c = 1.1f * ((float)D * EW * EW + 2.f * EW * P1);
    const float b2 = 1.1f * (2.f * sqrtf((float)D) * EW + 2.f * (gam + kU32) * P2);
    float T = INFINITY;
    int nc = 0;
    bool overflow = false;
    if (rs.box) {
      for (int a = 0; a < d; ++a) {
        float ua = 0.f;
        double ua64 = 0.0, va64 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k == a) {
            ua = u32[k];
            ua64 = u[k];
            va64 = v[k];
          }
        float tlo, thi;
        const int sd = face_bounds32(ua, ua64, __double2float_rn(va64), tlo, thi);
        if (sd < 0) continue;
        const int32_t fid = face_id(a, sd);
        bool ex = false;
        for (int q = 0; q < m; ++q) ex |= (eta[q] == fid);
        if (ex) continue;
        T = fminf(T, thi);
        if (nc < kCmax) {
          cid[nc] = fid;
          ctlo[nc] = tlo;
          ++nc;
        } else {
          overflow = true;
        }
      }
    }
    // reach of the ball of the current T and the squared-distance threshold
    // beyond which a list entry (and every later one) lies outside it
    float far2, wwx;
    bool stale = false;
    // Ball test of a finite bound T (Section 2.2's incircle criterion): with
    // w = x - g and q = p + T u, a node with den > 0 has t <= T exactly when
    // f = |w|^2 - 2 w.q <= 0.  In binary32 (w32 within EW per component,
    // q32 within EQ in norm, FMA chains within gam) f <= 0 implies
    //   fl(fl(cb ww32) - 2 wq32) <= beta,
    // cb = 1/(1+gam) - e1/(2 s0 (1-gam)) less two roundings, beta =
    // e1 s0/2 + e0, where e1 s + e0 bounds every error term with s = |w32|
    // (e1 = 2 gam Q + 2 sqrt(D) EW + 2 EQ + 4.03 u Q, e0 = D EW^2 +
    // 2 sqrt(D) EW (Q + EQ), Q >= |q32|) and s <= (s^2/s0 + s0)/2 with
    // s0 = Q.  A stale (larger) T gives a wider test, so it stays valid.
    float q32[D];
    float cb = 0.f, beta = 0.f;
    bool fast = false;
    auto refresh = [&]() {
      Ball<D> ball;
      make_ball<D>(g32, p32, u32, T, B, ball);
      far2 = far_radius2<D>(tr, ball, g32);
      wwx = ww_exit(far2, gam, EW, D);
      stale = false;
      fast = T < INFINITY;
      if (fast) {
        float Q2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          q32[k] = fmaf(T, u32[k], p32[k]);
          Q2 = fmaf(q32[k], q32[k], Q2);
        }
        const float Q = fmaxf(sqrtf(Q2) * (1.f + 2.f * gam), 0x1p-60f);
        const float EQ = 1.01f * kU32 * (Q + 1.0001f * T + P2) + 1e-37f;
        const float sD = sqrtf((float)D) * 1.0001f;
        const float e1 = 1.01f * (2.f * gam * Q + 2.f * sD * EW + 2.f * EQ + 4.03f * kU32 * Q);
        const float e0 = 1.01f * ((float)D * EW * EW + 2.f * sD * EW * (Q + EQ));
        const float c = (1.f - 1.01f * gam) - e1 / (2.f * Q * (1.f - gam)) * 1.0001f;
        cb = c - 2.02f * kU32 * fabsf(c) - 1e-30f;
        beta = (0.5f * e1 * Q + e0) * 1.001f + 1e-37f;
      }
    };
    refresh();
    // ---- list scan ----
    const int32_t* lst = tr.knn + (int64_t)g * tr.K;
    const int n = tr.kcnt[g];
    bool certified = false;
    int c = 0;
    // software pipeline: the next candidate's id and coordinates are loaded
    // while this one is screened, the id after that one further ahead
    int32_t nid = n > 0 ? lst[0] : 0;
    int32_t nnid = n > 1 ? lst[1] : 0;
    float xn[D];
    load_x32<D>(tr, nid, n > 0, xn);
    for (; c < n; ++c) {
      // a lowered T is used by the screening at once; the exit threshold
      // follows every fourth entry, in step on all lanes (a threshold from a
      // larger T is still valid: a node that can beat the smaller T lies in
      // the ball of the larger one; it only ends the scan a little later)
      if (stale && (c & 3) == 0) refresh();
      const int32_t id = nid;
      float xc[D];
#pragma unroll
      for (int k = 0; k < D; ++k) xc[k] = xn[k];
      nid = nnid;
      if (c + 2 < n) nnid = lst[c + 2];
      load_x32<D>(tr, nid, c + 1 < n, xn);
      float w[D];
      float ww = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        w[k] = (k < d) ? xc[k] - g32[k] : 0.f;
        ww = fmaf(w[k], w[k], ww);
      }
      if (ww >= wwx) {  // then true_d2_lower(ww) >= far2: this and every later node lie outside
        certified = true;
        break;
      }
      if (fast) {  // outside the ball of T: t >= T (or den <= 0), not a candidate
        float wq = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) wq = fmaf(w[k], q32[k], wq);
        if (fmaf(-2.f, wq, cb * ww) > beta) continue;
      }
      bool ok = true;  // the generators of eta are excluded by id
      for (int q = 0; q < m; ++q) ok &= (id != eta[q]);
      if (!ok) continue;
      float den = 0.f, pw = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) den = fmaf(u32[k], w[k], den);
      if (hasp) {
#pragma unroll
        for (int k = 0; k < D; ++k) pw = fmaf(p32[k], w[k], pw);
      }
      const float num = fmaf(-2.f, pw, ww);
      const float wn = norm_up(ww, gam);
      const float Eden = fmaf(a1, wn, a0);
      const float dh = den + Eden;
      if (!(dh > 0.f)) continue;
      const float Enum = fmaf(1.1f * kU32, fabsf(num), fmaf(1.1f * gam, ww, fmaf(b2, wn, b0c)));
      const float nlo = num - Enum;
      if (!(nlo <= 0.f || nlo <= 2.f * T * dh * (1.f + 8.f * kU32))) continue;
      const float dl = den - Eden;
      const float nhi = num + Enum;
      float thi = INFINITY, tlo = -INFINITY;
      if (dl > 0.f)
        thi = nhi >= 0.f ? __fdiv_rn(nhi, 2.f * dl) * (1.f + 4.f * kU32)
                         : __fdiv_rn(nhi, 2.f * dh) * (1.f - 4.f * kU32);
      if (nlo > 0.f) tlo = __fdiv_rn(nlo, 2.f * dh) * (1.f - 4.f * kU32);
      if (thi < T) {
        T = thi;
        stale = true;
      }
      if (!overflow && tlo <= T) {
        if (nc == kCmax) {  // drop entries the bound has excluded
          int k2 = 0;
          for (int q = 0; q < kCmax; ++q)
            if (ctlo[q] <= T) {
              cid[k2] = cid[q];
              ctlo[k2] = ctlo[q];
              ++k2;
            }
          nc = k2;
        }
        if (nc < kCmax) {
          cid[nc] = id;
          ctlo[nc] = tlo;
          ++nc;
        } else {
          overflow = true;
        }
      }
    }
    n_pairs += (unsigned)c;
    const int64_t op = out_pos(rs, ro, r);
    if (!certified) {
      if (stale) refresh();
      certified = true_d2_lower(tr.kcert[g], gam, EW, D) >= far2;
    }
    if (!certified) {  // finished by the tree walk, from the bound found so far
      const unsigned long long k = atomicAdd(&ctr->fallback, 1ull);
      if ((int64_t)k < ro.fallback_cap) ro.fallback_list[k] = (int32_t)r;
      else atomicOr(&ctr->flags, kFlagQueue);
      ro.t[op] = (double)T;
      continue;
    }
    if (overflow) {  // redone on the binary64 path
      const unsigned long long k = atomicAdd(&ctr->overflow, 1ull);
      if ((int64_t)k < ro.overflow_cap) ro.overflow_list[k] = (int32_t)r;
      else atomicOr(&ctr->flags, kFlagCandOverflow);
      ro.hit[op] = kNoId;
      ro.t[op] = NAN;
      continue;
    }
    // ---- binary64 recheck, canonical order ----
    load_vu<D>(tr, rs, r, v, u);  // loaded again rather than kept in registers through the scan
    double bt = INFINITY;
    int bc = 2, bk = 0;
    for (int q = 0; q < nc; ++q) {
      if (!(ctlo[q] <= T)) continue;
      const int32_t id = cid[q];
      ++n_rech;
      if (id >= 0) {
        double den = 0.0, ww = 0.0, pw = 0.0, w[D];
#pragma unroll
        for (int k = 0; k < D; ++k)
          w[k] = k < d ? __dadd_rn(tr.X[(int64_t)id * d + k], -tr.X[(int64_t)g * d + k]) : 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k < d) den = __dadd_rn(den, __dmul_rn(u[k], w[k]));
        if (!(den > 0.0)) continue;
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k < d) ww = __dadd_rn(ww, __dmul_rn(w[k], w[k]));
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k < d) pw = __dadd_rn(pw, __dmul_rn(__dadd_rn(v[k], -tr.X[(int64_t)g * d + k]), w[k]));
        const double num = __dadd_rn(ww, -__dmul_rn(2.0, pw));
        const double t = __ddiv_rn(num, __dmul_rn(2.0, den));
        if (better(t, 0, id, bt, bc, bk)) {
          bt = t;
          bc = 0;
          bk = id;
        }
      } else {
        const int a = face_axis(id), sd = face_side(id);
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
    }
    ro.hit[op] = gen_from_key(bc, bk);
    ro.t[op] = bt;
    if (ro.screen_err) ro.screen_err[op] = (bt > 0.0 && bt < INFINITY) ? (float)((T - bt) / bt) : 0.f;
  }
  unsigned long long sp = n_pairs, sr = n_rech;
  for (int o = 16; o; o >>= 1) {
    sp += __shfl_xor_sync(kFull, sp, o);
    sr += __shfl_xor_sync(kFull, sr, o);
  }
  if (lane == 0) {
    atomicAdd(&ctr->pairs, sp);
    atomicAdd(&ctr->rechecked, sr);
  }
}

// ------------------------------------------------------------------------
// VD_FP64: every pair in binary64, canonical order
// ------------------------------------------------------------------------
template <int D, bool LIST>
__global__ void __launch_bounds__(kWpb * 32) k_ray_fp64(TreeView tr, RaySource rs, RayOut ro, Counters* ctr,
                                                        unsigned long long* work, const int32_t* subset) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpF64<D>& S = reinterpret_cast<WarpF64<D>*>(smem_raw)[wib];
  const int d = tr.d;
  const float B = tr.coord_abs;
  const float gam = (float)(D + 1) * kU32 * 1.01f;
  const float EW = 4.01f * kU32 * B;
  unsigned long long n_tiles = 0, n_pairs = 0;
  int64_t R = rs.R;
  int rpb = rs.rpb;
  if (rs.R_dev) {
    R = min((int64_t)*rs.R_dev, rs.R);
    rpb = R < (int64_t)gridDim.x * kWpb * 64 ? 1 : 32;
  }
  while (true) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(work, 1ull);
    b = __shfl_sync(kFull, b, 0);
    const int64_t b0 = (int64_t)b * rpb;
    if (b0 >= R) break;
    const int64_t slot = b0 + lane;
    const bool vr = lane < rpb && slot < R;
    const int64_t r = vr ? (subset ? (int64_t)subset[slot] : slot) : 0;
    if (vr) {
      double v[D], u[D];
      int32_t eta[D + 1];
      int m;
      load_ray<D>(tr, rs, r, v, u, eta, m);
      if (m < 1 || eta[0] < 0 || eta[0] >= tr.N) {  // g must be a node
        atomicOr(&ctr->flags, kFlagBadInput);
        m = 1;
        eta[0] = 0;
      }
      const int32_t g = eta[0];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double gk = k < d ? tr.X[(int64_t)g * d + k] : 0.0;
        S.u[lane][k] = u[k];
        S.g[lane][k] = gk;
        S.p[lane][k] = __dadd_rn(v[k], -gk);
      }
      for (int q = 0; q <= D; ++q) S.eta[lane][q] = q < m ? eta[q] : kNoId;
      S.m[lane] = m;
      double bt = INFINITY;
      int bc = 2, bk = 0;
      if (rs.box) {
        for (int a = 0; a < d; ++a) {
          if (u[a] == 0.0) continue;
          const int s = u[a] > 0.0 ? 1 : 0;
          const int32_t fid = face_id(a, s);
          bool ex = false;
          for (int q = 0; q < m; ++q) ex |= (eta[q] == fid);
          if (ex) continue;
          const double t = __ddiv_rn(__dadd_rn(s ? 1.0 : 0.0, -v[a]), u[a]);
          if (better(t, 1, 2 * a + s, bt, bc, bk)) {
            bt = t;
            bc = 1;
            bk = 2 * a + s;
          }
        }
      }
      S.bt[lane] = bt;
      S.bcls[lane] = bc;
      S.bkey[lane] = bk;
    }
    __syncwarp();
    for (int rr = 0; rr < rpb && b0 + rr < R; ++rr) {
      double u[D], gg[D], pp[D];
      float u32[D], g32[D], p32[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        u[k] = S.u[rr][k];
        gg[k] = S.g[rr][k];
        pp[k] = S.p[rr][k];
        u32[k] = __double2float_rn(u[k]);
        g32[k] = __double2float_rn(gg[k]);
        p32[k] = __double2float_rn(pp[k]);
      }
      const int m = S.m[rr];
      double bt = S.bt[rr];
      int bc = S.bcls[rr], bk = S.bkey[rr];
      Ball<D> ball;
      make_ball<D>(g32, p32, u32, __double2float_ru(bt) * (1.f + 4.f * kU32), B, ball);
      auto eval = [&](int32_t id, const double* xs, int stride) {
        bool ok = id != kNoId;
        for (int q = 0; q < m; ++q) ok &= (id != S.eta[rr][q]);
        double w[D], den = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          w[k] = k < d ? __dadd_rn(xs[k * stride], -gg[k]) : 0.0;
          if (k < d) den = __dadd_rn(den, __dmul_rn(u[k], w[k]));
        }
        ok &= den > 0.0;
        double t = INFINITY;
        if (ok) {
          double ww = 0.0, pw = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k)
            if (k < d) ww = __dadd_rn(ww, __dmul_rn(w[k], w[k]));
#pragma unroll
          for (int k = 0; k < D; ++k)
            if (k < d) pw = __dadd_rn(pw, __dmul_rn(pp[k], w[k]));
          const double num = __dadd_rn(ww, -__dmul_rn(2.0, pw));
          // division only when the pair can reach the current best
          if (num <= 2.0 * bt * den * (1.0 + 0x1p-40)) t = __ddiv_rn(num, __dmul_rn(2.0, den));
        }
        const bool imp = ok && better(t, 0, id, bt, bc, bk);
        if (__ballot_sync(kFull, imp) == 0) return;
        double lt = imp ? t : bt;
        int lc = imp ? 0 : bc, lk = imp ? id : bk;
        warp_argmin(lt, lc, lk);
        bt = lt;
        bc = lc;
        bk = lk;
        make_ball<D>(g32, p32, u32, __double2float_ru(bt) * (1.f + 4.f * kU32), B, ball);
      };
      bool certified = true;
      if (!LIST) {
        auto leaf = [&](int64_t tile) {
          eval(tr.ids[tile * kTile + lane], tr.x64 + tile * d * kTile + lane, kTile);
        };
        unsigned long long t0 = n_tiles;
        walk<D>(tr, S.stk, ball, lane, leaf, n_tiles);
        n_pairs += (n_tiles - t0) * 32;
      } else {
        const int32_t g = S.eta[rr][0];
        const int32_t* lst = tr.knn + (int64_t)g * tr.K;
        const int n = tr.kcnt[g];
        certified = false;
        for (int c0 = 0; c0 < n; c0 += 32) {
          const int c = c0 + lane;
          const int32_t id = c < n ? lst[c] : kNoId;
          const int32_t ida = c < n ? id : g;
          eval(id, tr.X + (int64_t)ida * d, 1);
          n_pairs += 32;
          const float ww = ww32_of<D>(tr.X32 + (int64_t)ida * d, 1, g32, d);
          const float far2 = far_radius2<D>(tr, ball, g32);
          const bool far = c < n && true_d2_lower(ww, gam, EW, D) >= far2;
          if (__ballot_sync(kFull, far)) {
            certified = true;
            break;
          }
        }
        if (!certified) certified = true_d2_lower(tr.kcert[g], gam, EW, D) >= far_radius2<D>(tr, ball, g32);
      }
      if (lane == 0) {
        S.bt[rr] = bt;
        S.bcls[rr] = certified ? bc : -2;
        S.bkey[rr] = bk;
      }
      __syncwarp();
    }
    __syncwarp();
    if (vr) {
      const int64_t op = out_pos(rs, ro, r);
      if (S.bcls[lane] == -2) {
        const unsigned long long k = atomicAdd(&ctr->fallback, 1ull);
        if ((int64_t)k < ro.fallback_cap) ro.fallback_list[k] = (int32_t)r;
        else atomicOr(&ctr->flags, kFlagQueue);
      } else {
        ro.hit[op] = gen_from_key(S.bcls[lane], S.bkey[lane]);
        ro.t[op] = S.bt[lane];
        if (ro.screen_err) ro.screen_err[op] = 0.f;
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&ctr->tiles, n_tiles);
    atomicAdd(&ctr->pairs, n_pairs);
  }
}

template <int D>
__global__ void k_directions(uint64_t seed, uint32_t set, int64_t cell0, int64_t ncells, int64_t R, int d,
                             double* out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= ncells * R) return;
  const int64_t i = q / R, k = q % R;
  double u[D];
  mc_direction<D>(seed, set, (uint32_t)(cell0 + i), (uint32_t)k, d, u);
  for (int a = 0; a < d; ++a) out[q * d + a] = u[a];
}

template <int D>
cudaError_t launch_ray_d(const TreeView& tv, const RaySource& rs, const RayOut& ro, int precision, Counters* ctr,
                         unsigned long long* work, const int32_t* subset, int64_t nrays, bool list,
                         cudaStream_t st) {
  if (nrays <= 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  RaySource r2 = rs;
  r2.R = nrays;
  // few rays (the tree-walk leftovers of the list scan): one ray per warp so
  // that they spread over the SMs; otherwise 32 rays per warp
  r2.rpb = nrays < (int64_t)nsm * 256 ? 1 : 32;
  const int64_t batches = rs.R_dev ? (int64_t)nsm * 64 : (nrays + r2.rpb - 1) / r2.rpb;
  cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
  auto go = [&](auto kern, size_t sm) {
    allow_max_dyn_smem(kern);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWpb * 32, sm);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(occ, 1),
                                                                 (batches + kWpb - 1) / kWpb));
    kern<<<(unsigned)grid, kWpb * 32, sm, st>>>(tv, r2, ro, ctr, work, subset);
    count_launch();
  };
  if (precision == VD_FP64) {
    if (list) go(k_ray_fp64<D, true>, sizeof(WarpF64<D>) * kWpb);
    else go(k_ray_fp64<D, false>, sizeof(WarpF64<D>) * kWpb);
  } else if (list && subset == nullptr) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ray_list_thr<D>, kThrRays, 0);
    const int64_t want = rs.R_dev ? (int64_t)nsm * std::max(occ, 1) : (nrays + kThrRays - 1) / kThrRays;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(occ, 1), want));
    k_ray_list_thr<D><<<(unsigned)grid, kThrRays, 0, st>>>(tv, r2, ro, ctr, work);
    count_launch();
  } else {
    if (list) go(k_ray_mixed<D, true>, sizeof(WarpMixed<D>) * kWpb);
    else go(k_ray_mixed<D, false>, sizeof(WarpMixed<D>) * kWpb);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Candidate lists: for node g, the K nearest other nodes sorted by the
// binary32 squared distance ww32 (the same expression the list scan
// evaluates).  A warp gathers every node with ww32 <= r^2 by a tree walk
// (r adapted until more than K but at most `cap` nodes are found, or r
// covers all nodes), sorts them (bitonic, in shared memory), keeps K, and
// records kcert = the (K+1)-th smallest ww32 (or r^2): every node missing
// from the list has ww32 >= kcert.
// ------------------------------------------------------------------------
constexpr int kKnnCap = 2048;
constexpr int kKnnWpb = 4;

constexpr int kKnnTies = 64;

// One warp's shared memory: fixed part, then `cap` keys and `cap` ids (cap =
// the gather capacity of the launch, a power of two <= kKnnCap).
struct WarpKnn {
  int* stk;      // [kStk]
  int* hist;     // [256]
  int32_t* tie;  // [kKnnTies]
  float* key;    // [cap]
  int32_t* id;   // [cap]
};
constexpr size_t kKnnFixed = (sizeof(int) * (kStk + 256 + kKnnTies) + 15) / 16 * 16;
__host__ __device__ inline size_t knn_warp_bytes(int cap) { return kKnnFixed + (size_t)cap * 8; }
// Capacity of the gather for list length K: room for a ball about four
// times the list.
inline int knn_cap(int K) {
  int c = 256;
  while (c < 4 * K && c < kKnnCap) c <<= 1;
  return c;
}

// Bitonic sort of S.key/S.id[0, P) by (key, id), P a power of two.
__device__ __forceinline__ void knn_sort(WarpKnn& S, int P, int lane) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = lane; i < P / 2; i += 32) {
        const int lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const float ka = S.key[lo], kb = S.key[hi];
        const int32_t ia = S.id[lo], ib = S.id[hi];
        const bool gt = ka > kb || (ka == kb && ia > ib);
        if (asc == gt) {
          S.key[lo] = kb;
          S.key[hi] = ka;
          S.id[lo] = ib;
          S.id[hi] = ia;
        }
      }
      __syncwarp();
    }
  }
}

// Sort of S.key/S.id[0, n) by (key, id) with the buffer's second half
// S.key/S.id[n, 2n) as scratch (n <= cap / 2): a stable LSD radix sort by the
// key's bits (4 passes of 8 bits; non-negative floats order like their bit
// patterns; ranks among equal digits by __match_any_sync), then each run of
// equal keys ordered by id (ties are rare: lane 0 sorts them in place).
__device__ void knn_radix_sort(WarpKnn& S, int n, int lane) {
  const unsigned lt = (1u << lane) - 1u;
  float* kin = S.key;
  int32_t* iin = S.id;
  float* kout = S.key + n;
  int32_t* iout = S.id + n;
  for (int shift = 0; shift < 32; shift += 8) {
    for (int b = lane; b < 256; b += 32) S.hist[b] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) atomicAdd(&S.hist[(__float_as_uint(kin[i]) >> shift) & 255u], 1);
    __syncwarp();
    int c[8], tot = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = S.hist[lane * 8 + j];
      tot += c[j];
    }
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    int run = incl - tot;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      S.hist[lane * 8 + j] = run;
      run += c[j];
    }
    __syncwarp();
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int i = c0 + lane;
      const bool valid = i < n;
      const float k = valid ? kin[i] : 0.f;
      const int32_t id = valid ? iin[i] : 0;
      const int dg = valid ? (int)((__float_as_uint(k) >> shift) & 255u) : 256 + lane;
      const unsigned peers = __match_any_sync(kFull, dg);
      const int base = valid ? S.hist[dg] : 0;
      __syncwarp();
      if (valid) {
        const int pos = base + __popc(peers & lt);
        kout[pos] = k;
        iout[pos] = id;
        if (lane == __ffs(peers) - 1) S.hist[dg] = base + __popc(peers);
      }
      __syncwarp();
    }
    float* tk = kin;
    kin = kout;
    kout = tk;
    int32_t* ti = iin;
    iin = iout;
    iout = ti;
  }
  // four passes: the sorted keys are back in S.key/S.id[0, n)
  bool tie = false;
  for (int i = lane + 1; i < n; i += 32) tie |= S.key[i] == S.key[i - 1];
  if (__any_sync(kFull, tie) && lane == 0) {
    for (int i = 1; i < n; ++i) {
      const float k = S.key[i];
      const int32_t x = S.id[i];
      int j = i - 1;
      while (j >= 0 && S.key[j] == k && S.id[j] > x) {
        S.id[j + 1] = S.id[j];
        --j;
      }
      S.id[j + 1] = x;
    }
  }
  __syncwarp();
}

// Key of rank k (0-based) among S.key[0, n) (non-negative floats, whose bit
// patterns order like the values): most-significant-byte-first radix select.
__device__ __forceinline__ float knn_select(WarpKnn& S, int n, int k, int lane) {
  uint32_t prefix = 0, high = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = lane; b < 256; b += 32) S.hist[b] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const uint32_t bits = __float_as_uint(S.key[i]);
      if ((bits & high) == prefix) atomicAdd(&S.hist[(bits >> shift) & 255u], 1);
    }
    __syncwarp();
    int c[8], tot = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = S.hist[lane * 8 + j];
      tot += c[j];
    }
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - tot;
    const bool mine = k >= excl && k < incl;
    const unsigned who = __ballot_sync(kFull, mine);
    const int src = __ffs(who) - 1;
    int digit = 0, before = 0;
    if (mine) {
      int run = excl;
      for (int j = 0; j < 8; ++j) {
        if (k < run + c[j]) {
          digit = lane * 8 + j;
          before = run;
          break;
        }
        run += c[j];
      }
    }
    digit = __shfl_sync(kFull, digit, src);
    before = __shfl_sync(kFull, before, src);
    k -= before;
    prefix |= (uint32_t)digit << shift;
    high |= 255u << shift;
    __syncwarp();
  }
  return __uint_as_float(prefix);
}

template <int D>
__global__ void __launch_bounds__(kKnnWpb * 32) k_knn_build(TreeView tr, int K, int cap, float r0, float rmax,
                                                            int32_t* knn, int32_t* kcnt, float* kcert) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* wbase = smem_raw + knn_warp_bytes(cap) * wib;
  WarpKnn S;
  S.stk = reinterpret_cast<int*>(wbase);
  S.hist = S.stk + kStk;
  S.tie = S.hist + 256;
  S.key = reinterpret_cast<float*>(wbase + kKnnFixed);
  S.id = reinterpret_cast<int32_t*>(S.key + cap);
  const int d = tr.d;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t g = (int64_t)blockIdx.x * kKnnWpb + wib; g < tr.N; g += (int64_t)gridDim.x * kKnnWpb) {
    float g32[D];
#pragma unroll
    for (int k = 0; k < D; ++k) g32[k] = k < d ? tr.X32[g * d + k] : 0.f;
    float r = r0;
    {  // near the faces of the nodes' bounding box the ball holds fewer nodes:
       // one correction by the fraction of its bounding cube inside the box
      float f = 1.f;
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (k < d) {
          const float len = fminf(g32[k] + r, tr.root_hi[k]) - fmaxf(g32[k] - r, tr.root_lo[k]);
          f *= fmaxf(len, 1e-3f * r) / (2.f * r);
        }
      r = fminf(r * __powf(f, -1.f / (float)d), rmax);
    }
    int count = 0;
    const float target = fminf(1.5f * (float)K + 32.f, 0.75f * (float)cap);
    for (int attempt = 0; attempt < 64; ++attempt) {
      Ball<D> ball;
#pragma unroll
      for (int k = 0; k < D; ++k) ball.c[k] = g32[k];
      const float rho = r * (1.f + 8.f * (float)D * kU32) + 1e-30f;
      ball.rho_hi = rho;
      ball.lim2 = rho * rho * (1.f + 8.f * (float)D * kU32);
      const float r2 = r * r;
      count = 0;
      auto leaf = [&](int64_t tile) {
        const int32_t id = tr.ids[tile * kTile + lane];
        const float ww = ww32_of<D>(tr.x32 + tile * d * kTile + lane, kTile, g32, d);
        const bool in = id != kNoId && id != (int32_t)g && ww <= r2;
        const unsigned m = __ballot_sync(kFull, in);
        if (in) {
          const int pos = count + __popc(m & lt);
          if (pos < cap) {
            S.key[pos] = ww;
            S.id[pos] = id;
          }
        }
        count += __popc(m);
        __syncwarp();
      };
      walk_fixed<D>(tr, S.stk, ball, lane, leaf);
      // aim the ball at about `target` nodes: count scales like r^d
      if (count > cap) {
        r *= fminf(0.9f, __powf(target / (float)count, 1.f / (float)d));
        continue;
      }
      if (count <= K && r < rmax) {
        const float f = count > 0 ? __powf(target / (float)count, 1.f / (float)d) : 2.f;
        r = fminf(r * fminf(fmaxf(f, 1.1f), 2.f), rmax * 1.001f);
        continue;
      }
      break;
    }
    if (count > cap) {  // unresolvable (massive duplicates): no list, tree walk only
      if (lane == 0) {
        kcnt[g] = 0;
        kcert[g] = 0.f;
      }
      continue;
    }
    // keep the K smallest by (key, id): select the key of rank K, keep the
    // smaller keys and the smallest ids among the keys equal to it, then
    // sort only those K
    int n_sort = count;
    float cert = r * r;
    if (count > K) {
      const float tk = knn_select(S, count, K, lane);
      cert = tk;
      int nless = 0, ntie = 0;
      for (int c0 = 0; c0 < count; c0 += 32) {
        const int c = c0 + lane;
        const float kc = c < count ? S.key[c] : INFINITY;
        const int32_t ic = c < count ? S.id[c] : 0;
        const bool less = kc < tk, tie = kc == tk;
        const unsigned lm = __ballot_sync(kFull, less), tm = __ballot_sync(kFull, tie);
        __syncwarp();
        if (less) {
          const int pos = nless + __popc(lm & lt);
          S.key[pos] = kc;
          S.id[pos] = ic;
        }
        if (tie) {
          const int pos = ntie + __popc(tm & lt);
          if (pos < kKnnTies) S.tie[pos] = ic;
        }
        nless += __popc(lm);
        ntie += __popc(tm);
        __syncwarp();
      }
      const int need = K - nless;  // 1 <= need <= ntie
      if (ntie > kKnnTies) {       // massive ties: no list for this node, tree walk only
        if (lane == 0) {
          kcnt[g] = 0;
          kcert[g] = 0.f;
        }
        __syncwarp();
        continue;
      }
      if (lane == 0) {  // the need smallest ids among the ties (usually one)
        for (int a = 1; a < ntie; ++a) {
          const int32_t x = S.tie[a];
          int b = a - 1;
          while (b >= 0 && S.tie[b] > x) {
            S.tie[b + 1] = S.tie[b];
            --b;
          }
          S.tie[b + 1] = x;
        }
        for (int a = 0; a < need; ++a) {
          S.key[nless + a] = tk;
          S.id[nless + a] = S.tie[a];
        }
      }
      __syncwarp();
      n_sort = K;
    }
    if (2 * n_sort <= cap) {
      knn_radix_sort(S, n_sort, lane);
    } else {  // lists longer than half the gather buffer: bitonic sort in place
      int P = 1;
      while (P < n_sort) P <<= 1;
      for (int i = n_sort + lane; i < P; i += 32) {
        S.key[i] = INFINITY;
        S.id[i] = INT32_MAX;
      }
      __syncwarp();
      knn_sort(S, P, lane);
    }
    const int nk = min(count, K);
    for (int c = lane; c < nk; c += 32) knn[g * K + c] = S.id[c];
    if (lane == 0) {
      kcnt[g] = nk;
      kcert[g] = cert;
    }
    __syncwarp();
  }
}

__global__ void k_to_f32(const double* X, int64_t n, float* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = __double2float_rn(X[i]);
}

// out[i][j] = binary32 of X[i][j] for j < d, 0 for d <= j < 4q.
__global__ void k_to_f32v(const double* X, int64_t N, int d, int q, float* out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * q * 4) return;
  const int64_t i = t / (4 * q);
  const int j = (int)(t - i * 4 * q);
  out[t] = j < d ? __double2float_rn(X[i * d + j]) : 0.f;
}

template <int D>
cudaError_t launch_knn_d(TreeView* tv, int K, float r0, float rmax, int32_t* knn, int32_t* kcnt, float* kcert,
                         cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int cap = knn_cap(K);
  const size_t sm = knn_warp_bytes(cap) * kKnnWpb;
  allow_max_dyn_smem(k_knn_build<D>);  // batch preparation calls this from several threads
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_knn_build<D>, kKnnWpb * 32, sm);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(occ, 1) * 4,
                                                               (tv->N + kKnnWpb - 1) / kKnnWpb));
  k_knn_build<D><<<(unsigned)grid, kKnnWpb * 32, sm, st>>>(*tv, K, cap, r0, rmax, knn, kcnt, kcert);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

// Dimension dispatch: d is padded up to the next instantiated D (the padded
// coordinates are zero and contribute exact zeros to every sum).
#define VD_DISPATCH_D(d, FN, ...)              \
  ((d) <= 1   ? FN<1>(__VA_ARGS__)             \
   : (d) <= 2 ? FN<2>(__VA_ARGS__)             \
   : (d) <= 3 ? FN<3>(__VA_ARGS__)             \
   : (d) <= 4 ? FN<4>(__VA_ARGS__)             \
   : (d) <= 5 ? FN<5>(__VA_ARGS__)             \
   : (d) <= 6 ? FN<6>(__VA_ARGS__)             \
   : (d) <= 8 ? FN<8>(__VA_ARGS__)             \
   : (d) <= 12 ? FN<12>(__VA_ARGS__)           \
              : FN<16>(__VA_ARGS__))

cudaError_t launch_raycast(const TreeView& tv, const RaySource& rs, const RayOut& ro, int precision,
                           Counters* ctr, cudaStream_t st, int64_t* nfallback) {
  if (rs.R <= 0) return cudaSuccess;
  unsigned long long* work = reinterpret_cast<unsigned long long*>(&ctr->aux1);
  cudaError_t e;
  const bool list = tv.K > 0 && ro.fallback_list != nullptr;
  if (list) {
    cudaMemsetAsync(&ctr->fallback, 0, sizeof(unsigned long long), st);
    e = list_tc_ok(tv, rs, ro, precision)
            ? launch_list_tc(tv, rs, ro, ctr, st)
            : VD_DISPATCH_D(tv.d, launch_ray_d, tv, rs, ro, precision, ctr, work, nullptr, rs.R, true, st);
    if (e != cudaSuccess) return e;
    unsigned long long nfb = 0;
    cudaMemcpyAsync(&nfb, &ctr->fallback, sizeof(nfb), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    const int64_t n = std::min<int64_t>((int64_t)nfb, ro.fallback_cap);
    if (nfallback) *nfallback += n;
    if (n > 0) {
      RaySource rf = rs;
      rf.t_hint = 1;
      e = VD_DISPATCH_D(tv.d, launch_ray_d, tv, rf, ro, precision, ctr, work, ro.fallback_list, n, false, st);
    }
  } else {
    e = VD_DISPATCH_D(tv.d, launch_ray_d, tv, rs, ro, precision, ctr, work, nullptr, rs.R, false, st);
  }
  if (e != cudaSuccess || precision == VD_FP64) return e;
  // rays whose candidate list overflowed are redone on the binary64 path
  unsigned long long nover = 0;
  cudaMemcpyAsync(&nover, &ctr->overflow, sizeof(nover), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (nover > 0) {
    const int64_t n = std::min<int64_t>((int64_t)nover, ro.overflow_cap);
    e = VD_DISPATCH_D(tv.d, launch_ray_d, tv, rs, ro, VD_FP64, ctr, work, ro.overflow_list, n, false, st);
  }
  return e;
}

cudaError_t launch_raycast_async(const TreeView& tv, const RaySource& rs, const RayOut& ro, int precision,
                                 Counters* ctr, cudaStream_t st) {
  if (rs.R <= 0) return cudaSuccess;
  unsigned long long* work = reinterpret_cast<unsigned long long*>(&ctr->aux1);
  const bool list = tv.K > 0 && ro.fallback_list != nullptr;
  cudaError_t e = list_tc_ok(tv, rs, ro, precision)
                      ? launch_list_tc(tv, rs, ro, ctr, st)
                      : VD_DISPATCH_D(tv.d, launch_ray_d, tv, rs, ro, precision, ctr, work, nullptr, rs.R, list, st);
  if (e != cudaSuccess) return e;
  if (list) {  // rays the lists could not certify: tree walk, count on the device
    RaySource r2 = rs;
    r2.R = ro.fallback_cap;
    r2.R_dev = &ctr->fallback;
    r2.t_hint = 1;
    e = VD_DISPATCH_D(tv.d, launch_ray_d, tv, r2, ro, precision, ctr, work, ro.fallback_list, ro.fallback_cap,
                      false, st);
    if (e != cudaSuccess) return e;
  }
  if (precision == VD_FP64 || ro.overflow_list == nullptr) return cudaSuccess;
  RaySource r3 = rs;  // rays whose candidate buffer overflowed: binary64 path
  r3.R = ro.overflow_cap;
  r3.R_dev = &ctr->overflow;
  return VD_DISPATCH_D(tv.d, launch_ray_d, tv, r3, ro, VD_FP64, ctr, work, ro.overflow_list, ro.overflow_cap, false,
                       st);
}

cudaError_t launch_mc_fallback_dev(const SetDesc& S, int64_t R, uint64_t seed, cudaStream_t st) {
  TreeView tv = S.tv;
  tv.K = 0;  // tree walk
  RaySource rs;
  rs.mode = 1;
  rs.R = S.fb_cap;
  rs.R_dev = &S.ctr->fallback;
  rs.t_hint = 1;  // the cell kernel left each ray's bound in its output t
  rs.mc_cell = S.fb_cell;
  rs.mc_ray = S.fb_ray;
  rs.mc_rpc = R;
  rs.seed = seed;
  rs.set = S.set;
  rs.box = 1;
  RayOut ro;
  ro.hit = S.hit;
  ro.t = S.l;
  ro.mc_rpc = R;
  ro.overflow_list = S.ov_list;
  ro.overflow_cap = S.ov_cap;
  unsigned long long* work = reinterpret_cast<unsigned long long*>(&S.ctr->aux1);
  cudaError_t e = VD_DISPATCH_D(tv.d, launch_ray_d, tv, rs, ro, VD_FP32, S.ctr, work, nullptr, S.fb_cap, false, st);
  if (e != cudaSuccess) return e;
  RaySource r2 = rs;
  r2.R = S.ov_cap;
  r2.R_dev = &S.ctr->overflow;
  return VD_DISPATCH_D(tv.d, launch_ray_d, tv, r2, ro, VD_FP64, S.ctr, work, S.ov_list, S.ov_cap, false, st);
}

int default_knn_k(int d) {
  static const int k[] = {0, 16, 32, 96, 256, 1024, 1024, 1024, 1024};
  return d <= 8 ? k[d] : 0;
}

cudaError_t build_knn(TreeView* tv, int K, cudaStream_t st, DevBufs& bufs) {
  if (K <= 0) return cudaSuccess;
  const int d = tv->d;
  const int64_t N = tv->N;
  int32_t *knn = nullptr, *kcnt = nullptr;
  float *kcert = nullptr, *X32 = nullptr;
  cudaError_t e;
  if ((e = bufs.alloc_n(&knn, (size_t)N * K)) || (e = bufs.alloc_n(&kcnt, (size_t)N)) ||
      (e = bufs.alloc_n(&kcert, (size_t)N)) || (e = bufs.alloc_n(&X32, (size_t)N * d)))
    return e;
  k_to_f32<<<(unsigned)((N * d + 255) / 256), 256, 0, st>>>(tv->X, N * d, X32);
  count_launch();
  tv->X32 = X32;
  if (d <= 8) {  // the same coordinates in rows of 16-byte vectors, zero padded
    const int q = (d + 3) / 4;
    float4* X32v = nullptr;
    if ((e = bufs.alloc_n(&X32v, (size_t)N * q))) return e;
    k_to_f32v<<<(unsigned)((N * q * 4 + 255) / 256), 256, 0, st>>>(tv->X, N, d, q, reinterpret_cast<float*>(X32v));
    count_launch();
    tv->X32v = X32v;
    tv->x32q = q;
  }
  // initial radius: about 1.3 K nodes expected in the ball for the node
  // density of the bounding box of the root (the kernel corrects it per node
  // for the part of the ball outside that box)
  double vol = 1.0, diag2 = 0.0;
  {
    // the root's box is the nodes' bounding box the tree build read back
    const double* lo = tv->box_lo;
    const double* hi = tv->box_hi;
    for (int k = 0; k < d; ++k) {
      const double w = std::max(hi[k] - lo[k], 1e-12);
      vol *= w;
      diag2 += w * w;
      tv->root_lo[k] = std::nextafter((float)lo[k], -INFINITY);
      tv->root_hi[k] = std::nextafter((float)hi[k], INFINITY);
    }
  }
  const double vball = std::pow(M_PI, 0.5 * d) / std::tgamma(0.5 * d + 1.0);
  const float r0 = (float)std::pow(std::min(1.3 * K + 32, 0.75 * knn_cap(K)) * vol / ((double)N * vball), 1.0 / d);
  const float rmax = (float)std::sqrt(diag2) * 1.01f + 1e-6f;
  e = VD_DISPATCH_D(d, launch_knn_d, tv, K, std::min(r0, rmax), rmax, knn, kcnt, kcert, st);
  if (e != cudaSuccess) return e;
  tv->K = K;
  tv->knn = knn;
  tv->kcnt = kcnt;
  tv->kcert = kcert;
  return cudaStreamSynchronize(st);
}

cudaError_t launch_mc_directions(uint64_t seed, uint32_t set, int64_t cell0, int64_t ncells, int64_t R, int d,
                                 double* out, cudaStream_t st) {
  const int64_t n = ncells * R;
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 127) / 128);
#define VD_DIR(DD) k_directions<DD><<<grid, 128, 0, st>>>(seed, set, cell0, ncells, R, d, out)
  if (d <= 4) VD_DIR(4);
  else if (d <= 8) VD_DIR(8);
  else VD_DIR(16);
#undef VD_DIR
  count_launch();
  return cudaGetLastError();
}

}  // namespace vd
