// vd_traverse.cu -- exhaustive vertex traversal of the clipped Voronoi
// diagram (Section 2.3, Algorithm 2), frontier-parallel.
//
// Algorithm 2 pops one vertex at a time; here a whole BFS level is processed
// at once:
//   expand : for every frontier vertex sigma and edge eta = sigma \ {e} with
//            a node and edge counter G[eta] < 2, SearchDirection (binary64
//            null vector of the edge's constraint rows) -> one ray;
//   raycast: the generic RayCast kernels on the level's rays;
//   commit : sigma' = sort(eta + hit) is inserted into a device hash of
//            sorted generator tuples (two phases: claim a slot for the ray,
//            then give each winning ray a vertex id), its coordinates are
//            solved from the tuple in binary64, and G[eta'] += 1 for its
//            edges (device hash of sorted d-tuples).
// Seeds come from Descent (Algorithm 2): several nodes cast d rays each onto
// successively lower-dimensional faces.  The box faces are generators with
// negative ids, so no edge is unbounded.  The result is sorted into
// lexicographic tuple order.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "vd_dev.cuh"

namespace vd {

cudaError_t radix_sort_u64(uint64_t* keys, int32_t* vals, uint64_t* ktmp, int32_t* vtmp, int64_t n,
                           uint32_t* counts, unsigned long long* orand, cudaStream_t st);

namespace {

constexpr int32_t kEmpty = -1;
constexpr int32_t kRayTag = INT32_MIN;  // slot claimed by a ray during a level: kRayTag | ray
constexpr int kMaxProbe = 4096;

struct Tables {
  int d;
  // vertices
  int32_t* vt;       // [vcap][d+1]
  double* vx;        // [vcap][d]
  int64_t vcap;
  int32_t* vslot;    // [vhcap]
  int64_t vhmask;
  unsigned long long* nv;
  // edges
  int32_t* et;       // [ecap][d]
  int32_t* ecnt;     // [ecap]
  int64_t ecap;
  int32_t* eslot;    // [ehcap]
  int64_t ehmask;
  unsigned long long* ne;
  int edet;          // edge entries indexed v (d+1) + q (ecap >= vcap (d+1))
  // edges are counted and expanded only if they hold a node in [bc0, bc1)
  // (every node for the whole-diagram traversal; the current batch of
  // cells for the per-cell exploration)
  int32_t bc0, bc1;
};

__device__ __forceinline__ bool in_batch(const Tables& T, int32_t g) { return g >= T.bc0 && g < T.bc1; }

__device__ __forceinline__ uint64_t mix64(uint64_t h) {
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 33;
  return h;
}

__device__ __forceinline__ uint64_t hash_tuple(const int32_t* t, int L) {
  uint64_t h = 0x9E3779B97F4A7C15ull * (uint64_t)(L + 1);
  for (int q = 0; q < L; ++q) h = mix64(h ^ (uint64_t)(uint32_t)t[q] ^ ((uint64_t)q << 40));
  return h;
}

__device__ __forceinline__ bool tuple_eq(const volatile int32_t* a, const int32_t* b, int L) {
  for (int q = 0; q < L; ++q)
    if (a[q] != b[q]) return false;
  return true;
}

__device__ __forceinline__ void sort_small(int32_t* t, int L) {
  for (int a = 1; a < L; ++a) {
    const int32_t x = t[a];
    int b = a - 1;
    while (b >= 0 && t[b] > x) {
      t[b + 1] = t[b];
      --b;
    }
    t[b + 1] = x;
  }
}

// |x| rounded to binary32 (to nearest, ties to even) as an order-preserving
// integer, the bit pattern of that binary32 value, by integer operations (the
// same order as comparing __double2float_rn(fabs(x)), without the FP64-pipe
// conversion); kNanKey for NaN, which compares as no other key does.
constexpr int32_t kNanKey = INT32_MIN;
__device__ __forceinline__ int32_t f32key_abs(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  const int e = (int)(b >> 52);
  const uint64_t m = b & ((1ull << 52) - 1);
  if (e == 0x7FF) return m ? kNanKey : 0x7F800000;
  const int fe = e - 1023 + 127;
  if (fe <= 0) return __float_as_int(__double2float_rn(__longlong_as_double((long long)b)));  // zero or tiny
  if (fe >= 255) return 0x7F800000;
  uint32_t r = ((uint32_t)fe << 23) | (uint32_t)(m >> 29);
  const uint64_t rem = m & ((1ull << 29) - 1);
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (r & 1u))) r += 1u;  // a carry moves into the exponent
  return (int32_t)r;
}

// Canonical vertex coordinates from the sorted tuple (same steps as the
// definition: x0 = first node, y = r - x0, fixed axes from the faces,
// rows 2 w_k . y = |w_k|^2 on the free axes, partial pivoting with the
// magnitudes compared in binary32, multipliers through 1/pivot).
template <int D>
__device__ bool vertex_coords(const double* X, int d, const int32_t* sig, double* r) {
  int fixed[D], side[D];
  for (int a = 0; a < d; ++a) fixed[a] = 0;
  int nodes[D + 1], m = 0;
  for (int q = 0; q <= d; ++q) {
    if (sig[q] >= 0) {
      nodes[m++] = sig[q];
      continue;
    }
    const int a = face_axis(sig[q]);
    if (fixed[a]) return false;
    fixed[a] = 1;
    side[a] = face_side(sig[q]);
  }
  if (m < 1) return false;
  const double* x0 = X + (int64_t)nodes[0] * d;
  int freeax[D], nf = 0;
  double y[D];
  for (int a = 0; a < d; ++a) {
    if (fixed[a]) y[a] = __dadd_rn(side[a] ? 1.0 : 0.0, -x0[a]);
    else freeax[nf++] = a;
  }
  if (nf != m - 1) return false;
  double M[D][D], b[D];
  for (int rr = 0; rr < nf; ++rr) {
    const double* xk = X + (int64_t)nodes[rr + 1] * d;
    double w[D], ww = 0.0;
    for (int a = 0; a < d; ++a) w[a] = __dadd_rn(xk[a], -x0[a]);
    for (int a = 0; a < d; ++a) ww = __dadd_rn(ww, __dmul_rn(w[a], w[a]));
    for (int a = 0; a < d; ++a)
      if (fixed[a]) ww = __dadd_rn(ww, -__dmul_rn(__dmul_rn(2.0, w[a]), y[a]));
    for (int c = 0; c < nf; ++c) M[rr][c] = __dmul_rn(2.0, w[freeax[c]]);
    b[rr] = ww;
  }
  double inv[D];
  for (int c = 0; c < nf; ++c) {
    int piv = c;
    int32_t pbest = f32key_abs(M[c][c]);
    const bool pnan = pbest == kNanKey;  // a NaN magnitude compares below nothing
    for (int rr = c + 1; rr < nf; ++rr) {
      const int32_t a = f32key_abs(M[rr][c]);
      if (!pnan && a > pbest) {
        piv = rr;
        pbest = a;
      }
    }
    if (M[piv][c] == 0.0) return false;
    if (piv != c) {
      for (int cc = 0; cc < nf; ++cc) {
        const double tmp = M[c][cc];
        M[c][cc] = M[piv][cc];
        M[piv][cc] = tmp;
      }
      const double tb = b[c];
      b[c] = b[piv];
      b[piv] = tb;
    }
    inv[c] = __drcp_rn(M[c][c]);
    for (int rr = c + 1; rr < nf; ++rr) {
      const double f = __dmul_rn(M[rr][c], inv[c]);
      for (int cc = c + 1; cc < nf; ++cc) M[rr][cc] = __dadd_rn(M[rr][cc], -__dmul_rn(f, M[c][cc]));
      b[rr] = __dadd_rn(b[rr], -__dmul_rn(f, b[c]));
    }
  }
  double z[D];
  for (int c = nf - 1; c >= 0; --c) {
    double s = b[c];
    for (int cc = c + 1; cc < nf; ++cc) s = __dadd_rn(s, -__dmul_rn(M[c][cc], z[cc]));
    z[c] = __dmul_rn(s, inv[c]);
  }
  for (int c = 0; c < nf; ++c) y[freeax[c]] = z[c];
  for (int a = 0; a < d; ++a) r[a] = fixed[a] ? (side[a] ? 1.0 : 0.0) : __dadd_rn(x0[a], y[a]);
  return true;
}

// SearchDirection: unit null vector of the rows x_k - g (nodes of eta other
// than its first node g) on the axes not fixed by eta's faces; complete
// pivoting (first maximal |entry| in row-major order, magnitudes compared in
// binary32, multipliers through 1/pivot), the non-pivot column set to 1,
// back substitution, u = z * (1/|z|); sign so that the dropped node e has
// u.(x_e - g) < 0, a dropped lower face u_a > 0, an upper face u_a < 0.
template <int D>
__device__ bool search_direction(const double* X, int d, const int32_t* sig, int drop, double* u) {
  int32_t eta[D];
  int m = 0;
  for (int q = 0; q <= d; ++q)
    if (q != drop) eta[m++] = sig[q];
  int fixed[D];
  for (int a = 0; a < d; ++a) fixed[a] = 0;
  int nodes[D], mn = 0;
  for (int q = 0; q < d; ++q) {
    if (eta[q] >= 0) nodes[mn++] = eta[q];
    else fixed[face_axis(eta[q])] = 1;
  }
  if (mn < 1) return false;
  int freeax[D], nf = 0;
  for (int a = 0; a < d; ++a)
    if (!fixed[a]) freeax[nf++] = a;
  if (nf != mn) return false;
  const double* g = X + (int64_t)nodes[0] * d;
  const int nr = mn - 1;
  double M[D][D];
  for (int rr = 0; rr < nr; ++rr) {
    const double* xk = X + (int64_t)nodes[rr + 1] * d;
    for (int c = 0; c < nf; ++c) M[rr][c] = __dadd_rn(xk[freeax[c]], -g[freeax[c]]);
  }
  int colperm[D];
  for (int c = 0; c < nf; ++c) colperm[c] = c;
  double inv[D];
  for (int c = 0; c < nr; ++c) {
    int pr = c, pc = c;
    int32_t best = -1;  // below every magnitude (NaN has the lowest key)
    for (int rr = c; rr < nr; ++rr)
      for (int cc = c; cc < nf; ++cc) {
        const int32_t a = f32key_abs(M[rr][cc]);
        if (a > best) {
          best = a;
          pr = rr;
          pc = cc;
        }
      }
    if (M[pr][pc] == 0.0) return false;
    if (pr != c)
      for (int cc = 0; cc < nf; ++cc) {
        const double tmp = M[c][cc];
        M[c][cc] = M[pr][cc];
        M[pr][cc] = tmp;
      }
    if (pc != c) {
      for (int rr = 0; rr < nr; ++rr) {
        const double tmp = M[rr][c];
        M[rr][c] = M[rr][pc];
        M[rr][pc] = tmp;
      }
      const int tp = colperm[c];
      colperm[c] = colperm[pc];
      colperm[pc] = tp;
    }
    inv[c] = __drcp_rn(M[c][c]);
    for (int rr = c + 1; rr < nr; ++rr) {
      const double f = __dmul_rn(M[rr][c], inv[c]);
      for (int cc = c + 1; cc < nf; ++cc) M[rr][cc] = __dadd_rn(M[rr][cc], -__dmul_rn(f, M[c][cc]));
    }
  }
  double zp[D];
  zp[nf - 1] = 1.0;
  for (int c = nr - 1; c >= 0; --c) {
    double s = -M[c][nf - 1];
    for (int cc = c + 1; cc < nr; ++cc) s = __dadd_rn(s, -__dmul_rn(M[c][cc], zp[cc]));
    zp[c] = __dmul_rn(s, inv[c]);
  }
  double z[D];
  for (int c = 0; c < nf; ++c) z[colperm[c]] = zp[c];
  double nz = 0.0;
  for (int c = 0; c < nf; ++c) nz = __dadd_rn(nz, __dmul_rn(z[c], z[c]));
  const double invn = __drcp_rn(__dsqrt_rn(nz));
  for (int a = 0; a < d; ++a) u[a] = 0.0;
  for (int c = 0; c < nf; ++c) u[freeax[c]] = __dmul_rn(z[c], invn);
  const int32_t e = sig[drop];
  bool flip;
  if (e >= 0) {
    const double* xe = X + (int64_t)e * d;
    double den = 0.0;
    for (int a = 0; a < d; ++a) den = __dadd_rn(den, __dmul_rn(u[a], __dadd_rn(xe[a], -g[a])));
    if (den == 0.0) return false;
    flip = den > 0.0;
  } else {
    const int a = face_axis(e);
    if (u[a] == 0.0) return false;
    flip = face_side(e) ? (u[a] > 0.0) : (u[a] < 0.0);
  }
  if (flip)
    for (int a = 0; a < d; ++a) u[a] = -u[a];
  return true;
}

__device__ __forceinline__ int32_t vslot_load(const int32_t* p) { return *(const volatile int32_t*)p; }

// Looks up an edge counter; returns 0 if absent.
__device__ int edge_count(const Tables& T, const int32_t* eta) {
  const int L = T.d;
  uint64_t h = hash_tuple(eta, L) & (uint64_t)T.ehmask;
  for (int pr = 0; pr < kMaxProbe; ++pr) {
    const int32_t s = vslot_load(&T.eslot[h]);
    if (s == kEmpty) return 0;
    if (tuple_eq(T.et + (int64_t)s * L, eta, L)) return T.ecnt[s];
    h = (h + 1) & (uint64_t)T.ehmask;
  }
  return 0;
}

// G[eta] += 1, inserting eta if absent.  A new entry takes index `entry`
// (edge q of vertex v: v (d+1) + q, no shared counter) when entry >= 0, else
// the next index of the shared counter.
__device__ void edge_increment(const Tables& T, const int32_t* eta, int64_t entry, unsigned* flags) {
  const int L = T.d;
  uint64_t h = hash_tuple(eta, L) & (uint64_t)T.ehmask;
  int32_t mine = kEmpty;
  for (int pr = 0; pr < kMaxProbe; ++pr) {
    int32_t s = vslot_load(&T.eslot[h]);
    if (s == kEmpty) {
      if (mine == kEmpty) {
        const unsigned long long e = entry >= 0 ? (unsigned long long)entry : atomicAdd(T.ne, 1ull);
        if ((int64_t)e >= T.ecap) {
          atomicOr(flags, kFlagHashFull);
          return;
        }
        mine = (int32_t)e;
        for (int q = 0; q < L; ++q) T.et[(int64_t)mine * L + q] = eta[q];
        T.ecnt[mine] = 0;
        __threadfence();
      }
      s = atomicCAS(&T.eslot[h], kEmpty, mine);
      if (s == kEmpty) {
        atomicAdd(&T.ecnt[mine], 1);
        return;
      }
      __threadfence();
    }
    __threadfence();  // the entry's tuple was published before its slot
    if (tuple_eq(T.et + (int64_t)s * L, eta, L)) {
      atomicAdd(&T.ecnt[s], 1);
      return;  // our reserved entry (if any) stays unused
    }
    h = (h + 1) & (uint64_t)T.ehmask;
  }
  atomicOr(flags, kFlagHashFull);
}

// ---- level kernels ----------------------------------------------------------
// Warp-aggregated append: returns this lane's slot in a list whose length
// is *n (lanes with want == false get -1).
__device__ __forceinline__ long long warp_append(bool want, unsigned long long* n) {
  const unsigned m = __ballot_sync(__activemask(), want);
  if (!want) return -1;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(n, (unsigned long long)__popc(m));
  base = __shfl_sync(m, base, leader);
  return (long long)(base + __popc(m & ((1u << lane) - 1u)));
}

// Expansion, pass 1: every (frontier vertex, dropped generator) whose edge
// holds a node (of the batch) and has fewer than two known endpoints is
// appended to the level's work list (cheap hash lookups; pass 2 then runs the
// binary64 SearchDirection on full warps).  Frontier vertex f is f0 + f, or
// flist[f] when a list is given.
__global__ void k_expand_mark(Tables T, int64_t f0, const int32_t* flist, int64_t nf, int64_t* items,
                              unsigned long long* nitems, int64_t rcap, unsigned* flags) {
  const int d = T.d;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool want = false;
  if (q < nf * (d + 1)) {
    const int64_t f = q / (d + 1);
    const int drop = (int)(q % (d + 1));
    const int64_t v = flist ? (int64_t)flist[f] : f0 + f;
    int32_t eta[VD_MAX_D];
    int m = 0, hasnode = 0;
    for (int a = 0; a <= d; ++a)
      if (a != drop) {
        const int32_t g = T.vt[(int64_t)v * (d + 1) + a];
        eta[m++] = g;
        hasnode |= in_batch(T, g);
      }
    want = hasnode && edge_count(T, eta) < 2;
  }
  const long long r = warp_append(want, nitems);
  if (r < 0) return;
  if (r >= rcap) {
    atomicOr(flags, kFlagQueue);
    return;
  }
  items[r] = q;
}

// Expansion, pass 2: ray r of the level from the r-th work item: origin =
// the vertex, direction = SearchDirection, eta = the edge (reference node
// first).
template <int D>
__global__ void k_expand_dir(Tables T, const double* X, int64_t f0, const int32_t* flist, const int64_t* items,
                             const unsigned long long* nitems, int64_t rcap, double* ro, double* rd, int32_t* reta,
                             unsigned* flags) {
  const int d = T.d;
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= min(rcap, (int64_t)*nitems)) return;
  const int64_t q = items[r];
  const int64_t f = q / (d + 1);
  const int drop = (int)(q % (d + 1));
  const int64_t v = flist ? (int64_t)flist[f] : f0 + f;
  int32_t sig[D + 1], eta[D];
  for (int a = 0; a <= d; ++a) sig[a] = T.vt[(int64_t)v * (d + 1) + a];
  int m = 0;
  for (int a = 0; a <= d; ++a)
    if (a != drop) eta[m++] = sig[a];
  double u[D];
  if (!search_direction<D>(X, d, sig, drop, u)) {
    atomicOr(flags, kFlagDegenerate);
    for (int a = 0; a < d; ++a) u[a] = 0.0;  // casts to nothing; the commit flags it again
  }
  // eta row: reference node g (first node of eta) first
  int gpos = 0;
  while (eta[gpos] < 0) ++gpos;
  reta[r * d + 0] = eta[gpos];
  int k = 1;
  for (int a = 0; a < d; ++a)
    if (a != gpos) reta[r * d + k++] = eta[a];
  for (int a = 0; a < d; ++a) {
    ro[r * d + a] = T.vx[(int64_t)v * d + a];
    rd[r * d + a] = u[a];
  }
}

// Phase 1 of the commit: claim the tuple's slot for ray r (or find it);
// true if this ray owns a new vertex.
// A seed that reached no vertex (Descent gave up on it) arrives with hit =
// kNoId and is skipped when no_hit_ok is set; on a traversal level a ray
// without a hit is a degenerate input.
__device__ bool claim_slot(const Tables& T, const int32_t* reta, const int32_t* hit, int64_t r, int32_t* cand,
                           int64_t* cslot, unsigned* flags, bool no_hit_ok) {
  const int d = T.d, L = d + 1;
  int32_t sig[VD_MAX_D + 1];
  for (int a = 0; a < d; ++a) sig[a] = reta[r * d + a];
  sig[d] = hit[r];
  cslot[r] = -1;
  if (sig[d] == kNoId) {
    if (!no_hit_ok) atomicOr(flags, kFlagDegenerate);
    return false;
  }
  sort_small(sig, L);
  for (int a = 0; a < L; ++a) cand[r * L + a] = sig[a];
  __threadfence();
  uint64_t h = hash_tuple(sig, L) & (uint64_t)T.vhmask;
  for (int pr = 0; pr < kMaxProbe; ++pr) {
    int32_t s = vslot_load(&T.vslot[h]);
    if (s == kEmpty) {
      s = atomicCAS(&T.vslot[h], kEmpty, kRayTag | (int32_t)r);
      if (s == kEmpty) {
        cslot[r] = (int64_t)h;  // this ray owns the new vertex
        return true;
      }
      __threadfence();
    }
    __threadfence();  // the other ray's tuple was published before its claim
    const volatile int32_t* other = (s & kRayTag) ? (cand + (int64_t)(s & ~kRayTag) * L) : (T.vt + (int64_t)s * L);
    if (tuple_eq(other, sig, L)) return false;  // known vertex or claimed by another ray
    h = (h + 1) & (uint64_t)T.vhmask;
  }
  atomicOr(flags, kFlagHashFull);
  return false;
}

// Rays that own a new vertex are appended to win[] (count *nwin).
__global__ void k_commit_claim(Tables T, const int32_t* reta, const int32_t* hit, int64_t nr,
                               const unsigned long long* nr_dev, int32_t* cand, int64_t* cslot, int32_t* win,
                               unsigned long long* nwin, unsigned* flags, int seeds) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool owns =
      r < (nr_dev ? min(nr, (int64_t)*nr_dev) : nr) && claim_slot(T, reta, hit, r, cand, cslot, flags, seeds != 0);
  const long long p = warp_append(owns, nwin);
  if (p >= 0) win[p] = (int32_t)r;
}

// Phase 2: winners get vertex ids, coordinates, frontier slots and edges.
// New vertex ids are consecutive, so the next frontier is the id range the
// level added.
template <int D>
__global__ void k_commit_finish(Tables T, const double* X, const int32_t* cand, const int64_t* cslot,
                                const int32_t* win, int64_t nwcap, const unsigned long long* nwin, int32_t* vids,
                                unsigned* flags) {
  const int d = T.d, L = d + 1;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= min(nwcap, (int64_t)*nwin)) return;
  const int64_t r = win[p];
  const long long v = warp_append(true, T.nv);
  if ((int64_t)v >= T.vcap) {
    atomicOr(flags, kFlagHashFull);
    vids[p] = -1;
    return;
  }
  int32_t sig[D + 1];
  for (int a = 0; a < L; ++a) sig[a] = cand[r * L + a];
  for (int a = 0; a < L; ++a) T.vt[(int64_t)v * L + a] = sig[a];
  double x[D];
  if (!vertex_coords<D>(X, d, sig, x)) atomicOr(flags, kFlagDegenerate);
  for (int a = 0; a < d; ++a) T.vx[(int64_t)v * d + a] = x[a];
  __threadfence();
  T.vslot[cslot[r]] = (int32_t)v;
  vids[p] = (int32_t)v;
}

// Edge counters of the level's new vertices: one thread per (vertex, edge),
// so the dependent hash probes of the d + 1 edges run side by side.
__global__ void k_commit_edges(Tables T, const int32_t* vids, int64_t nwcap, const unsigned long long* nwin,
                               unsigned* flags) {
  const int d = T.d, L = d + 1;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p = t / L;
  const int q = (int)(t % L);
  if (p >= min(nwcap, (int64_t)*nwin)) return;
  const int32_t v = vids[p];
  if (v < 0) return;
  int32_t eta[VD_MAX_D];
  int m = 0, hasnode = 0;
  for (int a = 0; a <= d; ++a)
    if (a != q) {
      const int32_t g = T.vt[(int64_t)v * L + a];
      eta[m++] = g;
      hasnode |= in_batch(T, g);
    }
  if (hasnode) edge_increment(T, eta, T.edet ? (int64_t)v * L + q : -1, flags);
}

// ---- per-cell exploration (Section 2.3: cells explored in sequential order,
// the edge counts reconstructed for the current cells only) ----
// Start of a batch of cells [bc0, bc1), one thread per (known vertex, edge):
// the counters of the edges that hold a batch node, the known vertices with a
// batch node (the batch's first frontier, in flist) and the batch cells that
// already have a vertex (hasv).
__global__ void k_cell_recount(Tables T, int64_t nv, int32_t* flist, unsigned long long* nfl, int32_t* hasv,
                               unsigned* flags) {
  const int d = T.d, L = d + 1;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nv * L) return;
  const int64_t v = t / L;
  const int q = (int)(t % L);
  const int32_t* sig = T.vt + v * L;
  int32_t eta[VD_MAX_D];
  int m = 0;
  bool eb = false, vb = false;
  for (int a = 0; a <= d; ++a) {
    const int32_t g = sig[a];
    const bool b = in_batch(T, g);
    vb |= b;
    if (a != q) {
      eta[m++] = g;
      eb |= b;
    }
  }
  if (eb) edge_increment(T, eta, -1, flags);
  if (q == 0 && vb)
    for (int a = 0; a <= d; ++a)
      if (in_batch(T, sig[a])) hasv[sig[a] - T.bc0] = 1;
  const long long p = warp_append(q == 0 && vb, nfl);
  if (p >= 0) flist[p] = (int32_t)v;
}

// flist[base + k] = a + k for the vertex ids a .. b - 1 (a batch's seeds).
__global__ void k_append_range(int32_t* flist, int64_t base, int64_t a, int64_t b) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a + k < b) flist[base + k] = (int32_t)(a + k);
}

// Marks the batch cells with a vertex among the ids a .. b - 1.
__global__ void k_cell_mark(Tables T, int64_t a, int64_t b, int32_t* hasv) {
  const int L = T.d + 1;
  const int64_t v = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= b) return;
  for (int q = 0; q < L; ++q) {
    const int32_t g = T.vt[v * L + q];
    if (in_batch(T, g)) hasv[g - T.bc0] = 1;
  }
}

// ---- Descent seeding ----------------------------------------------------------
// Seed s starts at node nodes[s] with sigma = {node}, r = x_node; each step
// draws a direction (the MC generator on set 0xFFFFFFFF, cell = node, ray =
// step), removes its components along the span of the current constraint
// rows (x_k - g for the other nodes, e_a for faces; modified Gram-Schmidt),
// and casts a ray with eta = sigma.
__global__ void k_descent_dir(const double* X, int d, int64_t ns, const int32_t* snode, const int32_t* ssig,
                              const int* sm, const double* sr, int step, double* ro, double* rd, int32_t* reta,
                              int* alive) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= ns) return;
  // a dead seed still casts a valid ray (its result is ignored)
  for (int a = 0; a < d; ++a) {
    ro[s * d + a] = X[(int64_t)snode[s] * d + a];
    rd[s * d + a] = a == 0 ? 1.0 : 0.0;
  }
  reta[s * (d + 1)] = snode[s];
  for (int k = 1; k <= d; ++k) reta[s * (d + 1) + k] = kNoId;
  if (!alive[s]) return;
  const int m = sm[s];
  const int32_t* sig = ssig + s * (VD_MAX_D + 1);
  double u[VD_MAX_D];
  mc_direction<VD_MAX_D>(0x5EEDull, 0xFFFFFFFFu, (uint32_t)snode[s], (uint32_t)step, d, u);
  int32_t g = -1;
  for (int q = 0; q < m; ++q)
    if (sig[q] >= 0 && (g < 0 || sig[q] < g)) g = sig[q];
  double B[VD_MAX_D + 1][VD_MAX_D];
  int nb = 0;
  for (int q = 0; q < m; ++q) {
    if (sig[q] == g) continue;
    if (sig[q] >= 0)
      for (int a = 0; a < d; ++a) B[nb][a] = X[(int64_t)sig[q] * d + a] - X[(int64_t)g * d + a];
    else {
      for (int a = 0; a < d; ++a) B[nb][a] = 0.0;
      B[nb][face_axis(sig[q])] = 1.0;
    }
    ++nb;
  }
  for (int q = 0; q < nb; ++q) {
    for (int q2 = 0; q2 < q; ++q2) {
      double dp = 0.0;
      for (int a = 0; a < d; ++a) dp += B[q][a] * B[q2][a];
      for (int a = 0; a < d; ++a) B[q][a] -= dp * B[q2][a];
    }
    double nn = 0.0;
    for (int a = 0; a < d; ++a) nn += B[q][a] * B[q][a];
    nn = sqrt(nn);
    if (nn == 0.0) {
      alive[s] = 0;
      return;
    }
    for (int a = 0; a < d; ++a) B[q][a] /= nn;
  }
  for (int q = 0; q < nb; ++q) {
    double dp = 0.0;
    for (int a = 0; a < d; ++a) dp += u[a] * B[q][a];
    for (int a = 0; a < d; ++a) u[a] -= dp * B[q][a];
  }
  for (int q = 0; q < m; ++q)
    if (sig[q] < 0) u[face_axis(sig[q])] = 0.0;
  double nu = 0.0;
  for (int a = 0; a < d; ++a) nu += u[a] * u[a];
  nu = sqrt(nu);
  if (!(nu > 1e-12)) {
    alive[s] = 0;
    return;
  }
  for (int a = 0; a < d; ++a) {
    rd[s * d + a] = u[a] / nu;
    ro[s * d + a] = sr[s * VD_MAX_D + a];
  }
  int k = 1;
  reta[s * (d + 1) + 0] = g;
  for (int q = 0; q < m; ++q)
    if (sig[q] != g) reta[s * (d + 1) + k++] = sig[q];
  for (; k <= d; ++k) reta[s * (d + 1) + k] = kNoId;
}

__global__ void k_descent_update(int d, int64_t ns, int32_t* ssig, int* sm, double* sr, const double* rd,
                                 const int32_t* hit, const double* t, int* alive) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= ns || !alive[s]) return;
  if (hit[s] == kNoId || !(t[s] < INFINITY)) {
    alive[s] = 0;
    return;
  }
  for (int a = 0; a < d; ++a) sr[s * VD_MAX_D + a] += t[s] * rd[s * d + a];
  ssig[s * (VD_MAX_D + 1) + sm[s]] = hit[s];
  sm[s] += 1;
}

// Seeds that reached d+1 generators become rays of a pseudo level: their
// tuples are inserted like the commit of a level (cand rows and claim).
__global__ void k_descent_cand(int d, int64_t ns, const int32_t* ssig, const int* sm, const int* alive,
                               int32_t* reta, int32_t* hit) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= ns) return;
  if (!alive[s] || sm[s] != d + 1) {
    hit[s] = kNoId;
    for (int a = 0; a < d; ++a) reta[s * d + a] = kNoId;
    return;
  }
  for (int a = 0; a < d; ++a) reta[s * d + a] = ssig[s * (VD_MAX_D + 1) + a];
  hit[s] = ssig[s * (VD_MAX_D + 1) + d];
}

// The level's counters (nv, ne, rays, -, winners), the tree-walk and binary64
// follow-up counts and the flags, written to mapped host memory.
__global__ void k_read_level(const unsigned long long* cnts, const Counters* ctr, volatile unsigned long long* out) {
  const int t = threadIdx.x;
  if (t < 5) out[t] = cnts[t];
  else if (t == 5) out[5] = ctr->fallback;
  else if (t == 6) out[6] = ctr->overflow;
  else if (t == 7) out[7] = ctr->flags;
}

// Seed s at node snode[s]: sigma = {node}, one generator, alive, r = x_node.
__global__ void k_seed_init(const double* X, int d, int64_t ns, const int32_t* snode, int32_t* ssig, int* sm,
                            int* alive, double* sr) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= ns) return;
  ssig[s * (VD_MAX_D + 1)] = snode[s];
  for (int k = 1; k <= VD_MAX_D; ++k) ssig[s * (VD_MAX_D + 1) + k] = kNoId;
  sm[s] = 1;
  alive[s] = 1;
  for (int a = 0; a < VD_MAX_D; ++a) sr[s * VD_MAX_D + a] = a < d ? X[(int64_t)snode[s] * d + a] : 0.0;
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_iota(int32_t* p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

// keys[i] = tuple columns c0 .. c1 of vertex perm[i], each shifted by `off`
// to be non-negative and packed `bits` wide, column c0 most significant.
__global__ void k_col_keys(const int32_t* vt, int L, int c0, int c1, int bits, int32_t off, const int32_t* perm,
                           int64_t n, uint64_t* keys, int32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t v = perm[i];
  uint64_t k = 0;
  for (int c = c0; c <= c1; ++c) k = (k << bits) | (uint64_t)(uint32_t)(vt[(int64_t)v * L + c] + off);
  keys[i] = k;
  vals[i] = v;
}

__global__ void k_gather_out(const int32_t* vt, const double* vx, int d, const int32_t* perm, int64_t n,
                             int32_t* ot, double* ox) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t v = perm[i];
  for (int a = 0; a <= d; ++a) ot[i * (d + 1) + a] = vt[(int64_t)v * (d + 1) + a];
  for (int a = 0; a < d; ++a) ox[i * d + a] = vx[(int64_t)v * d + a];
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// The level's rays: nf frontier vertices -> work list -> ray arrays (count
// *nrays on the device, at most min(nf (d+1), rcap)).
template <int D>
void launch_expand(Tables T, const double* X, int64_t f0, const int32_t* flist, int64_t nf, int64_t* items,
                   double* ro, double* rd, int32_t* reta, unsigned long long* nrays, int64_t rcap, unsigned* flags,
                   cudaStream_t st) {
  const int64_t n = nf * (T.d + 1);
  k_expand_mark<<<nb(n), 256, 0, st>>>(T, f0, flist, nf, items, nrays, rcap, flags);
  count_launch();
  k_expand_dir<D><<<nb(std::min(n, rcap), 128), 128, 0, st>>>(T, X, f0, flist, items, nrays, rcap, ro, rd, reta,
                                                                flags);
  count_launch();
}

template <int D>
void launch_finish(Tables T, const double* X, const int32_t* cand, const int64_t* cslot, const int32_t* win,
                   int64_t nwcap, const unsigned long long* nwin, int32_t* vids, unsigned* flags, cudaStream_t st) {
  k_commit_finish<D><<<nb(nwcap), 256, 0, st>>>(T, X, cand, cslot, win, nwcap, nwin, vids, flags);
  count_launch();
  k_commit_edges<<<nb(nwcap * (T.d + 1)), 256, 0, st>>>(T, vids, nwcap, nwin, flags);
  count_launch();
}

#define VD_TRAV_D(d, FN, ...)                 \
  do {                                        \
    if ((d) <= 2) FN<2>(__VA_ARGS__);         \
    else if ((d) <= 3) FN<3>(__VA_ARGS__);    \
    else if ((d) <= 4) FN<4>(__VA_ARGS__);    \
    else if ((d) <= 5) FN<5>(__VA_ARGS__);    \
    else if ((d) <= 6) FN<6>(__VA_ARGS__);    \
    else if ((d) <= 8) FN<8>(__VA_ARGS__);    \
    else FN<16>(__VA_ARGS__);                 \
  } while (0)

// ---- random walks on the vertex graph (Section 2.3) ----
// Walker w at the vertex with sorted tuple sig[w] takes one of its edges that
// hold a node: with the valid drop indices a_0 < ... < a_{n-1} it takes a_k,
// k = (w0 n) >> 32, w0 = word 0 of Philox4x32-10 at counter (step, w,
// 0x57414C4B, 0), key (seed); the ray along that edge (SearchDirection from
// the vertex, reference node first) finds the far vertex sort(edge + hit).
template <int D>
__global__ void k_walk_init(const double* X, int d, int64_t W, const int32_t* sig, double* r, unsigned* flags) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= W) return;
  int32_t s[D + 1];
  for (int a = 0; a <= d; ++a) s[a] = sig[w * (d + 1) + a];
  double x[D];
  if (!vertex_coords<D>(X, d, s, x)) atomicOr(flags, kFlagDegenerate);
  for (int a = 0; a < d; ++a) r[w * d + a] = x[a];
}

template <int D>
__global__ void k_walk_dir(const double* X, int d, int64_t W, const int32_t* sig, const double* r, int64_t step,
                           uint64_t seed, double* ro, double* rd, int32_t* reta, int32_t* drop_out, unsigned* flags) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int L = d + 1;
  int32_t s[D + 1];
  for (int a = 0; a < L; ++a) s[a] = sig[w * L + a];
  int valid[D + 1], n = 0;
  for (int q = 0; q < L; ++q) {
    bool node = false;
    for (int k = 0; k < L; ++k) node |= (k != q && s[k] >= 0);
    if (node) valid[n++] = q;
  }
  int drop = -1;
  if (n > 0) {
    uint32_t c[4] = {(uint32_t)step, (uint32_t)w, 0x57414C4Bu, 0u};
    philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    drop = valid[(int)(((uint64_t)c[0] * (uint64_t)n) >> 32)];
  }
  double u[D];
  for (int a = 0; a < D; ++a) u[a] = 0.0;
  if (drop >= 0 && !search_direction<D>(X, d, s, drop, u)) {
    atomicOr(flags, kFlagDegenerate);
    for (int a = 0; a < D; ++a) u[a] = 0.0;
    drop = -1;
  }
  // eta row: the edge, reference node first (a zero direction casts to nothing)
  int32_t eta[D + 1];
  int m = 0;
  for (int a = 0; a < L; ++a)
    if (a != (drop >= 0 ? drop : 0)) eta[m++] = s[a];
  int gpos = 0;
  while (gpos < d && eta[gpos] < 0) ++gpos;
  if (gpos == d) {  // no node: not a vertex of this node set
    atomicOr(flags, kFlagDegenerate);
    drop = -1;
    reta[w * d] = 0;
    for (int a = 1; a < d; ++a) reta[w * d + a] = kNoId;
  } else {
    reta[w * d] = eta[gpos];
    int k = 1;
    for (int a = 0; a < d; ++a)
      if (a != gpos) reta[w * d + k++] = eta[a];
  }
  for (int a = 0; a < d; ++a) {
    ro[w * d + a] = r[w * d + a];
    rd[w * d + a] = u[a];
  }
  drop_out[w] = drop;
}

template <int D>
__global__ void k_walk_commit(const double* X, int d, int64_t W, int32_t* sig, double* r, const int32_t* drop,
                              const int32_t* hit, int64_t step, int64_t S, int32_t* path_t, double* path_x,
                              unsigned* flags) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int L = d + 1;
  int32_t s[D + 1];
  for (int a = 0; a < L; ++a) s[a] = sig[w * L + a];
  const int dr = drop[w];
  const int32_t h = hit[w];
  bool ok = dr >= 0 && h != kNoId;
  if (ok) {
    int32_t ns[D + 1];
    int m = 0;
    for (int a = 0; a < L; ++a)
      if (a != dr) ns[m++] = s[a];
    ns[d] = h;
    sort_small(ns, L);
    double x[D];
    ok = vertex_coords<D>(X, d, ns, x);
    if (ok) {
      for (int a = 0; a < L; ++a) sig[w * L + a] = s[a] = ns[a];
      for (int a = 0; a < d; ++a) r[w * d + a] = x[a];
    }
  }
  if (!ok) atomicOr(flags, kFlagDegenerate);  // the walker stays where it was
  for (int a = 0; a < L; ++a) path_t[(w * S + step) * L + a] = s[a];
  if (path_x)
    for (int a = 0; a < d; ++a) path_x[(w * S + step) * d + a] = r[w * d + a];
}

template <int D>
void walk_init_d(const double* X, int d, int64_t W, const int32_t* sig, double* r, unsigned* flags, cudaStream_t st) {
  k_walk_init<D><<<nb(W, 128), 128, 0, st>>>(X, d, W, sig, r, flags);
  count_launch();
}

template <int D>
void walk_dir_d(const double* X, int d, int64_t W, const int32_t* sig, const double* r, int64_t step, uint64_t seed,
                double* ro, double* rd, int32_t* reta, int32_t* drop, unsigned* flags, cudaStream_t st) {
  k_walk_dir<D><<<nb(W, 128), 128, 0, st>>>(X, d, W, sig, r, step, seed, ro, rd, reta, drop, flags);
  count_launch();
}

template <int D>
void walk_commit_d(const double* X, int d, int64_t W, int32_t* sig, double* r, const int32_t* drop,
                   const int32_t* hit, int64_t step, int64_t S, int32_t* path_t, double* path_x, unsigned* flags,
                   cudaStream_t st) {
  k_walk_commit<D><<<nb(W, 128), 128, 0, st>>>(X, d, W, sig, r, drop, hit, step, S, path_t, path_x, flags);
  count_launch();
}

int64_t pow2_at_least(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

// Expected vertices per cell (uniform nodes) for sizing, from the paper's
// table of vertices per cell (d = 2..7) extended by a factor d+2 per
// dimension.
static double vertices_per_cell(int d) {
  static const double t[] = {2, 2, 6.6, 29.2, 191, 1250, 9720, 91900};
  if (d <= 7) return t[d];
  double v = t[7];
  for (int k = 8; k <= d; ++k) v *= (k + 2);
  return v;
}

cudaError_t traverse_vertices(const TreeView& tv, int precision, const vd_config& cfg, int64_t cells_per_batch,
                              Workspace& ws, DevBufs& out_bufs, int32_t** tuples_out, double** coords_out,
                              int64_t* nv_out, vd_stats* stats, Counters* ctr, cudaStream_t st, char* err,
                              size_t errlen) {
  const int d = tv.d;
  const int L = d + 1;
  const int64_t N = tv.N;
  cudaError_t e;
#define VD_TRY(x)                     \
  do {                                \
    e = (x);                          \
    if (e != cudaSuccess) return e;   \
  } while (0)
  // workspace slots
  enum {
    kVt, kVx, kVslot, kEt, kEcnt, kEslot, kCnts, kRo, kRd, kRt, kReta, kRhit, kCand, kCslot, kOvl, kFbl, kSnode,
    kSsig, kSm, kAlive, kSr, kPerm, kPtmp, kKeys, kKtmp, kCounts, kOrand, kItems, kWin, kVids, kGrp, kFlist, kHasv
  };
  int64_t vcap = cfg.hash_capacity > 0 ? cfg.hash_capacity
                                       : (int64_t)std::min(2.0e9, std::max(1.0e5, 2.0 * N * vertices_per_cell(d) / L +
                                                                                       64.0 * (1 << std::min(d, 16)) +
                                                                                       8.0 * N * d));
  vcap = std::min<int64_t>(vcap, (int64_t)1 << 30);
  // expected edges ~ V (d+1) / 2; entries indexed v (d+1) + q while that fits.
  // The per-cell exploration holds only the edges of one batch of cells: each
  // cell has ~d/2 edges per vertex (edges of cell i hold i)
  const int64_t B = cells_per_batch > 0 ? std::min<int64_t>(cells_per_batch, N) : 0;
  int64_t ehint = std::min<int64_t>((int64_t)1 << 30, vcap * L / 2 + vcap / 4 + 1024);
  if (B > 0)
    ehint = std::min<int64_t>(ehint, (int64_t)std::min(1.0e9, (double)B * vertices_per_cell(d) * d + 65536.0));
  const bool edet = B == 0 && vcap * L < ((int64_t)1 << 31);
  const int64_t ecap = edet ? vcap * L : ehint;
  const int64_t vh = pow2_at_least(2 * vcap), eh = pow2_at_least(2 * ehint);
  Tables T;
  T.d = d;
  T.vcap = vcap;
  T.ecap = ecap;
  T.edet = edet ? 1 : 0;
  T.bc0 = 0;
  T.bc1 = INT32_MAX;
  T.vhmask = vh - 1;
  T.ehmask = eh - 1;
  VD_TRY(ws.get_n(kVt, (size_t)vcap * L, &T.vt));
  VD_TRY(ws.get_n(kVx, (size_t)vcap * d, &T.vx));
  VD_TRY(ws.get_n(kVslot, (size_t)vh, &T.vslot));
  VD_TRY(ws.get_n(kEt, (size_t)ecap * d, &T.et));
  VD_TRY(ws.get_n(kEcnt, (size_t)ecap, &T.ecnt));
  VD_TRY(ws.get_n(kEslot, (size_t)eh, &T.eslot));
  unsigned long long* cnts = nullptr;  // nv, ne, nrays, (unused), nwin, frontier list length
  VD_TRY(ws.get_n(kCnts, 6, &cnts));
  T.nv = cnts + 0;
  T.ne = cnts + 1;
  unsigned* flags = &ctr->flags;
  VD_TRY(cudaMemsetAsync(cnts, 0, 6 * sizeof(unsigned long long), st));
  k_fill_i32<<<nb(vh), 256, 0, st>>>(T.vslot, vh, kEmpty); count_launch();
  k_fill_i32<<<nb(eh), 256, 0, st>>>(T.eslot, eh, kEmpty); count_launch();

  // per-level ray buffers (contents live for one level; grown between levels)
  int64_t rcap = 0;
  double *ro = nullptr, *rd = nullptr, *rt = nullptr;
  int32_t *reta = nullptr, *rhit = nullptr, *cand = nullptr;
  int64_t *cslot = nullptr, *items = nullptr;
  int32_t *ovl = nullptr, *fbl = nullptr, *win = nullptr, *vids = nullptr, *grp = nullptr;
  int64_t grp_ints = 0;
  auto grow = [&](int64_t need) -> cudaError_t {
    if (need <= rcap) return cudaSuccess;
    const int64_t c = std::max<int64_t>({need, rcap * 2, 4096});
    cudaError_t ee;
    if ((ee = ws.get_n(kRo, (size_t)c * d, &ro)) || (ee = ws.get_n(kRd, (size_t)c * d, &rd)) ||
        (ee = ws.get_n(kRt, (size_t)c, &rt)) || (ee = ws.get_n(kReta, (size_t)c * L, &reta)) ||
        (ee = ws.get_n(kRhit, (size_t)c, &rhit)) || (ee = ws.get_n(kCand, (size_t)c * L, &cand)) ||
        (ee = ws.get_n(kCslot, (size_t)c, &cslot)) || (ee = ws.get_n(kOvl, (size_t)c, &ovl)) ||
        (ee = ws.get_n(kFbl, (size_t)c, &fbl)) || (ee = ws.get_n(kItems, (size_t)c, &items)) ||
        (ee = ws.get_n(kWin, (size_t)c, &win)) || (ee = ws.get_n(kVids, (size_t)c, &vids)))
      return ee;
    if (precision == VD_TC16) {  // grouping scratch of the tensor-core list RayCast
      grp_ints = grp_ray_ints(N, c);
      if ((ee = ws.get_n(kGrp, (size_t)grp_ints, &grp))) return ee;
    }
    rcap = c;
    return cudaSuccess;
  };
  // the widest level of a traversal holds a small fraction of all vertices
  VD_TRY(grow(std::min<int64_t>(vcap * L, std::max<int64_t>(4096, vcap * L / 16))));
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  double raycast_ms = 0.0;
  int64_t nfallback = 0, noverflow = 0;
  // casts the level's rays (count on the device if nr_dev != nullptr, at most nr)
  auto cast = [&](int64_t nr, const unsigned long long* nr_dev, int stride) -> cudaError_t {
    RaySource rs;
    rs.mode = 0;
    rs.R = nr;
    rs.R_dev = nr_dev;
    rs.origins = ro;
    rs.dirs = rd;
    rs.eta = reta;
    rs.eta_stride = stride;
    rs.box = 1;
    rs.wait_limit = cfg.wait_limit;
    RayOut rout;
    rout.hit = rhit;
    rout.t = rt;
    rout.overflow_list = ovl;
    rout.overflow_cap = rcap;
    rout.fallback_list = fbl;
    rout.fallback_cap = rcap;
    rout.grp_buf = grp;
    rout.grp_ints = grp_ints;
    cudaError_t ee = cudaMemsetAsync(&ctr->overflow, 0, sizeof(unsigned long long), st);
    if (ee == cudaSuccess) ee = cudaMemsetAsync(&ctr->fallback, 0, sizeof(unsigned long long), st);
    if (ee != cudaSuccess) return ee;
    cudaEventRecord(ev0, st);
    ee = launch_raycast_async(tv, rs, rout, precision, ctr, st);
    cudaEventRecord(ev1, st);
    return ee;
  };
  // after the stream has been synchronised
  auto account = [&](const unsigned long long* fb_host) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) raycast_ms += ms;
    nfallback += (int64_t)std::min<unsigned long long>(*fb_host, (unsigned long long)rcap);
  };

  unsigned long long* nrays = cnts + 2;
  unsigned long long* nwin = cnts + 4;
  int64_t raycasts = 0, levels = 0;
  int64_t nv_known = 0;  // vertices in the table (host copy)
  bool stop = false;     // a flag that ends the call was raised
  auto read_nv = [&]() -> cudaError_t {
    unsigned long long h = 0;
    cudaError_t ee = cudaMemcpyAsync(&h, cnts, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
    nv_known = std::min<int64_t>((int64_t)h, vcap);
    return ee;
  };

  // ---- Descent (Algorithm 2): nodes -> seed vertices, committed like a level ----
  int32_t *snode = nullptr, *ssig = nullptr;
  int *sm = nullptr, *alive = nullptr;
  double* sr = nullptr;
  auto descent = [&](const std::vector<int32_t>& nodes) -> cudaError_t {
    const int64_t ns = (int64_t)nodes.size();
    if (ns == 0) return cudaSuccess;
    cudaError_t ee;
    if ((ee = grow(ns)) || (ee = ws.get_n(kSnode, ns, &snode)) ||
        (ee = ws.get_n(kSsig, (size_t)ns * (VD_MAX_D + 1), &ssig)) || (ee = ws.get_n(kSm, ns, &sm)) ||
        (ee = ws.get_n(kAlive, ns, &alive)) || (ee = ws.get_n(kSr, (size_t)ns * VD_MAX_D, &sr)) ||
        (ee = cudaMemcpyAsync(snode, nodes.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice, st)))
      return ee;
    k_seed_init<<<nb(ns, 64), 64, 0, st>>>(tv.X, d, ns, snode, ssig, sm, alive, sr); count_launch();
    for (int step = 0; step < d; ++step) {
      k_descent_dir<<<nb(ns, 64), 64, 0, st>>>(tv.X, d, ns, snode, ssig, sm, sr, step, ro, rd, reta, alive);
      count_launch();
      if ((ee = cudaGetLastError()) || (ee = cast(ns, nullptr, L))) return ee;
      raycasts += ns;
      k_descent_update<<<nb(ns, 64), 64, 0, st>>>(d, ns, ssig, sm, sr, rd, rhit, rt, alive); count_launch();
    }
    k_descent_cand<<<nb(ns, 64), 64, 0, st>>>(d, ns, ssig, sm, alive, reta, rhit); count_launch();
    if ((ee = cudaMemsetAsync(nwin, 0, sizeof(unsigned long long), st))) return ee;
    // seeds that did not reach a vertex carry hit = kNoId and are skipped (a
    // missing seed is not an error); every other flag stays as raised
    k_commit_claim<<<nb(ns), 256, 0, st>>>(T, reta, rhit, ns, nullptr, cand, cslot, win, nwin, flags, 1);
    count_launch();
    VD_TRAV_D(d, launch_finish, T, tv.X, cand, cslot, win, ns, nwin, vids, flags, st);
    if ((ee = cudaGetLastError())) return ee;
    return read_nv();
  };

  // ---- BFS levels from a frontier (the id range f0 .. f0 + nf - 1, or the
  // first nf ids of fl); one host synchronisation per expansion; a level's new
  // vertices (consecutive ids) are the next frontier.  A frontier wider than
  // `slice` vertices is expanded in slices. ----
  const int64_t max_levels = cfg.max_levels > 0 ? cfg.max_levels : (int64_t)1 << 20;
  auto run_levels = [&](int64_t f0, int64_t nf, const int32_t* fl, int64_t slice) -> cudaError_t {
    cudaError_t ee;
    while (nf > 0 && !stop) {
      if (levels >= max_levels) {
        snprintf(err, errlen, "traversal stopped at the level cap %lld", (long long)max_levels);
        return cudaErrorUnknown;
      }
      ++levels;
      const int64_t level_start = nv_known;
      for (int64_t s0 = 0; s0 < nf && !stop; s0 += slice) {
        const int64_t nfs = std::min(slice, nf - s0);
        const int64_t ncap = nfs * L;  // at most one ray per (frontier vertex, edge)
        if ((ee = grow(ncap)) || (ee = cudaMemsetAsync(cnts + 2, 0, 3 * sizeof(unsigned long long), st))) return ee;
        VD_TRAV_D(d, launch_expand, T, tv.X, fl ? 0 : f0 + s0, fl ? fl + s0 : nullptr, nfs, items, ro, rd, reta,
                  nrays, rcap, flags, st);
        if ((ee = cudaGetLastError())) return ee;
        const int64_t rmax = std::min(ncap, rcap);
        if ((ee = cast(rmax, nrays, d))) return ee;
        k_commit_claim<<<nb(rmax), 256, 0, st>>>(T, reta, rhit, rmax, nrays, cand, cslot, win, nwin, flags, 0);
        count_launch();
        VD_TRAV_D(d, launch_finish, T, tv.X, cand, cslot, win, rmax, nwin, vids, flags, st);
        if ((ee = cudaGetLastError())) return ee;
        unsigned long long* hw = nullptr;
        if ((ee = ws.host_words_get(&hw))) return ee;
        k_read_level<<<1, 32, 0, st>>>(cnts, ctr, hw);
        count_launch();
        if ((ee = cudaGetLastError()) || (ee = cudaStreamSynchronize(st))) return ee;
        const volatile unsigned long long* hv = hw;
        unsigned long long hc[6];
        for (int k = 0; k < 4; ++k) hc[k] = hv[k];
        hc[4] = hv[5];
        hc[5] = hv[6];
        const unsigned hf = (unsigned)hv[7];
        account(hc + 4);
        noverflow += (int64_t)std::min<unsigned long long>(hc[5], (unsigned long long)rcap);
        raycasts += (int64_t)std::min<unsigned long long>(hc[2], (unsigned long long)rcap);
        nv_known = std::min<int64_t>((int64_t)hc[0], vcap);
        if (hf & (kFlagHashFull | kFlagQueue | kFlagDegenerate | kFlagCandOverflow | kFlagBadInput)) stop = true;
      }
      nf = nv_known - level_start;
      f0 = level_start;
      fl = nullptr;
    }
    return cudaSuccess;
  };

  if (B == 0) {
    // whole diagram: seeds at 64 nodes spread over the index range
    const int64_t ns = std::min<int64_t>(N, 64);
    std::vector<int32_t> hn(ns);
    for (int64_t s = 0; s < ns; ++s) hn[s] = (int32_t)((s * N) / ns);
    VD_TRY(descent(hn));
    if (nv_known == 0) {
      snprintf(err, errlen, "Descent found no seed vertex");
      return cudaErrorUnknown;
    }
    VD_TRY(run_levels(0, nv_known, nullptr, INT64_MAX));
  } else {
    // per cell, batches of B cells in index order: the edge table is rebuilt
    // for each batch from the vertices known so far, batch cells without a
    // known vertex are seeded by Descent, and the BFS follows only edges that
    // hold a batch node (both ends of such an edge are vertices of that cell)
    int32_t *flist = nullptr, *hasv = nullptr;
    VD_TRY(ws.get_n(kFlist, (size_t)vcap, &flist));
    VD_TRY(ws.get_n(kHasv, (size_t)B, &hasv));
    unsigned long long* nfl = cnts + 5;
    const int64_t slice = std::max<int64_t>(4096, rcap / L);
    std::vector<int32_t> hv(B);
    for (int64_t c0 = 0; c0 < N && !stop; c0 += B) {
      const int64_t c1 = std::min<int64_t>(N, c0 + B), nb_cells = c1 - c0;
      T.bc0 = (int32_t)c0;
      T.bc1 = (int32_t)c1;
      k_fill_i32<<<nb(eh), 256, 0, st>>>(T.eslot, eh, kEmpty); count_launch();
      VD_TRY(cudaMemsetAsync(T.ne, 0, sizeof(unsigned long long), st));
      VD_TRY(cudaMemsetAsync(nfl, 0, sizeof(unsigned long long), st));
      VD_TRY(cudaMemsetAsync(hasv, 0, (size_t)nb_cells * sizeof(int32_t), st));
      if (nv_known > 0) {
        k_cell_recount<<<nb(nv_known * L), 256, 0, st>>>(T, nv_known, flist, nfl, hasv, flags); count_launch();
      }
      unsigned long long hn_fl = 0;
      VD_TRY(cudaMemcpyAsync(hv.data(), hasv, (size_t)nb_cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      VD_TRY(cudaMemcpyAsync(&hn_fl, nfl, sizeof(hn_fl), cudaMemcpyDeviceToHost, st));
      VD_TRY(cudaStreamSynchronize(st));
      std::vector<int32_t> seeds;
      for (int64_t k = 0; k < nb_cells; ++k)
        if (!hv[k]) seeds.push_back((int32_t)(c0 + k));
      const int64_t batch_start = nv_known;
      VD_TRY(descent(seeds));
      const int64_t nfirst = (int64_t)hn_fl + (nv_known - batch_start);
      if (nv_known > batch_start) {
        k_append_range<<<nb(nv_known - batch_start), 256, 0, st>>>(flist, (int64_t)hn_fl, batch_start, nv_known);
        count_launch();
      }
      VD_TRY(run_levels(0, nfirst, flist, slice));
      if (stop) break;
      // every batch cell must have been reached
      if (nv_known > batch_start) {
        k_cell_mark<<<nb(nv_known - batch_start), 256, 0, st>>>(T, batch_start, nv_known, hasv); count_launch();
      }
      VD_TRY(cudaMemcpyAsync(hv.data(), hasv, (size_t)nb_cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      VD_TRY(cudaStreamSynchronize(st));
      for (int64_t k = 0; k < nb_cells; ++k)
        if (!hv[k]) {
          snprintf(err, errlen, "per-cell exploration reached no vertex of cell %lld", (long long)(c0 + k));
          return cudaErrorUnknown;
        }
    }
  }
  unsigned long long hc[4];
  VD_TRY(cudaMemcpyAsync(hc, cnts, sizeof(hc), cudaMemcpyDeviceToHost, st));
  VD_TRY(cudaStreamSynchronize(st));
  const int64_t nv = std::min<int64_t>((int64_t)hc[0], vcap);
  // lexicographic order: stable LSD sort by the tuple columns, last first
  int32_t *perm = nullptr, *ptmp = nullptr;
  uint64_t *keys = nullptr, *ktmp = nullptr;
  uint32_t* counts = nullptr;
  unsigned long long* orand = nullptr;
  const int64_t nvv = std::max<int64_t>(nv, 1);
  VD_TRY(ws.get_n(kPerm, nvv, &perm));
  VD_TRY(ws.get_n(kPtmp, nvv, &ptmp));
  VD_TRY(ws.get_n(kKeys, nvv, &keys));
  VD_TRY(ws.get_n(kKtmp, nvv, &ktmp));
  VD_TRY(ws.get_n(kCounts, (size_t)256 * (nvv / 4096 + 2), &counts));
  VD_TRY(ws.get_n(kOrand, 2, &orand));
  k_iota<<<nb(nvv), 256, 0, st>>>(perm, nv); count_launch();
  // ids + (2d + 1) lie in [0, N + 2d + 1): pack as many columns per 64-bit key
  // as fit and sort the groups of columns last to first (stable LSD)
  const int32_t off = 2 * d + 1;
  int bits = 1;
  while (((int64_t)1 << bits) < N + off) ++bits;
  const int per = std::max(1, 64 / bits);
  for (int c1 = d; c1 >= 0; c1 -= per) {
    const int c0 = std::max(0, c1 - per + 1);
    k_col_keys<<<nb(nvv), 256, 0, st>>>(T.vt, L, c0, c1, bits, off, perm, nv, keys, ptmp); count_launch();
    VD_TRY(radix_sort_u64(keys, ptmp, ktmp, perm, nv, counts, orand, st));
    VD_TRY(cudaMemcpyAsync(perm, ptmp, nv * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  }
  int32_t* ot = nullptr;
  double* ox = nullptr;
  VD_TRY(out_bufs.alloc_n(&ot, (size_t)nvv * L));
  VD_TRY(out_bufs.alloc_n(&ox, (size_t)nvv * d));
  k_gather_out<<<nb(nvv), 256, 0, st>>>(T.vt, T.vx, d, perm, nv, ot, ox); count_launch();
  VD_TRY(cudaStreamSynchronize(st));
  VD_TRY(cudaGetLastError());
  *tuples_out = ot;
  *coords_out = ox;
  *nv_out = nv;
  stats->levels = levels;
  stats->vertices = nv;
  stats->rays = raycasts;
  stats->raycast_ms = raycast_ms;
  stats->fallback_rays = nfallback;
  stats->overflow_rays = noverflow;
  stats->edge_table_bytes = ecap * (int64_t)(d + 1) * (int64_t)sizeof(int32_t) + eh * (int64_t)sizeof(int32_t);
  stats->vertex_table_bytes =
      vcap * (int64_t)(L * sizeof(int32_t) + d * sizeof(double)) + vh * (int64_t)sizeof(int32_t);
  return cudaSuccess;
#undef VD_TRY
}

// W walkers from the vertices start (device, W x (d+1) sorted tuples), S
// steps each; path_t (W x S x (d+1)) and path_x (W x S x d, may be null) on
// the device.  Flags (degenerate steps, bad input) go to ctr->flags.
cudaError_t random_walk(const TreeView& tv, int precision, const int32_t* start, int64_t W, int64_t S, uint64_t seed,
                        int32_t* path_t, double* path_x, Counters* ctr, DevBufs& scratch, cudaStream_t st,
                        double* raycast_ms) {
  const int d = tv.d, L = d + 1;
  const int64_t w1 = std::max<int64_t>(W, 1);
  int32_t *sig = nullptr, *reta = nullptr, *rhit = nullptr, *drop = nullptr, *ovl = nullptr, *fbl = nullptr,
          *grp = nullptr;
  const int64_t grp_ints = precision == VD_TC16 ? grp_ray_ints(tv.N, w1) : 0;
  double *r = nullptr, *ro = nullptr, *rd = nullptr, *rt = nullptr;
  cudaError_t e;
  if ((e = scratch.alloc_n(&sig, (size_t)w1 * L)) || (e = scratch.alloc_n(&r, (size_t)w1 * d)) ||
      (e = scratch.alloc_n(&ro, (size_t)w1 * d)) || (e = scratch.alloc_n(&rd, (size_t)w1 * d)) ||
      (e = scratch.alloc_n(&reta, (size_t)w1 * d)) || (e = scratch.alloc_n(&rhit, (size_t)w1)) ||
      (e = scratch.alloc_n(&rt, (size_t)w1)) || (e = scratch.alloc_n(&drop, (size_t)w1)) ||
      (e = scratch.alloc_n(&ovl, (size_t)w1)) || (e = scratch.alloc_n(&fbl, (size_t)w1)) ||
      (grp_ints > 0 && (e = scratch.alloc_n(&grp, (size_t)grp_ints))))
    return e;
  if (W == 0 || S == 0) return cudaSuccess;
  if ((e = cudaMemcpyAsync(sig, start, (size_t)W * L * sizeof(int32_t), cudaMemcpyDeviceToDevice, st))) return e;
  unsigned* flags = &ctr->flags;
  VD_TRAV_D(d, walk_init_d, tv.X, d, W, sig, r, flags, st);
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  float total = 0.f;
  for (int64_t step = 0; step < S && e == cudaSuccess; ++step) {
    VD_TRAV_D(d, walk_dir_d, tv.X, d, W, sig, r, step, seed, ro, rd, reta, drop, flags, st);
    RaySource rs;
    rs.mode = 0;
    rs.R = W;
    rs.origins = ro;
    rs.dirs = rd;
    rs.eta = reta;
    rs.eta_stride = d;
    rs.box = 1;
    RayOut rout;
    rout.hit = rhit;
    rout.t = rt;
    rout.overflow_list = ovl;
    rout.overflow_cap = W;
    rout.fallback_list = fbl;
    rout.fallback_cap = W;
    rout.grp_buf = grp;
    rout.grp_ints = grp_ints;
    if ((e = cudaMemsetAsync(&ctr->overflow, 0, sizeof(unsigned long long), st)) ||
        (e = cudaMemsetAsync(&ctr->fallback, 0, sizeof(unsigned long long), st)))
      break;
    cudaEventRecord(ev0, st);
    e = launch_raycast_async(tv, rs, rout, precision, ctr, st);
    cudaEventRecord(ev1, st);
    if (e != cudaSuccess) break;
    VD_TRAV_D(d, walk_commit_d, tv.X, d, W, sig, r, drop, rhit, step, S, path_t, path_x, flags, st);
    if ((e = cudaEventSynchronize(ev1)) == cudaSuccess) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) total += ms;
    }
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (raycast_ms) *raycast_ms = total;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace vd
