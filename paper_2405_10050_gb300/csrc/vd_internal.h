// vd_internal.h -- host/device structures shared by the libvd translation
// units (node tree, ray batches, counters, launcher prototypes).
#pragma once
#include <atomic>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "vd.h"

namespace vd {

constexpr int kTile = 32;      // nodes per leaf tile (one per lane)
constexpr int kFan = 32;       // children per internal tree node
constexpr int kMaxLev = 8;     // tree levels (leaves + internal)
constexpr int32_t kNoId = INT32_MIN;

// Device error flags (bit mask in Counters::flags).
enum : uint32_t {
  kFlagCandOverflow = 1u,   // a ray's candidate list overflowed (ray rerun on FP64)
  kFlagStack = 2u,          // traversal stack overflow
  kFlagHashFull = 4u,       // vertex / edge table full
  kFlagTimeout = 8u,        // bounded wait gave up
  kFlagDegenerate = 16u,    // degenerate solve or exact tie
  kFlagQueue = 32u,         // a work queue overflowed
  kFlagBadInput = 64u,      // a ray's reference generator is not a node
};

// Morton-ordered node tiles with a bounding-box hierarchy.
struct TreeView {
  int d = 0;
  int64_t N = 0;
  int64_t ntiles = 0;
  int nlev = 0;                 // number of levels, level 0 = tiles, level nlev-1 = root (1 node)
  int64_t cnt[kMaxLev] = {};    // nodes per level
  int64_t off[kMaxLev] = {};    // first index of each level in the bbox arrays
  int64_t total = 0;            // bbox entries over all levels
  const float* blo32 = nullptr;  // [d][total], rounded down
  const float* bhi32 = nullptr;  // [d][total], rounded up
  const double* blo64 = nullptr; // [d][total]
  const double* bhi64 = nullptr;
  const float* rho32 = nullptr;  // [total] radius of the node's points around its binary32 box centre
  const float* x32 = nullptr;    // [ntiles][d][32], nearest binary32 of x
  const double* x64 = nullptr;   // [ntiles][d][32]
  const int32_t* ids = nullptr;  // [ntiles][32], kNoId for padding
  const double* X = nullptr;     // original N x d row-major
  float coord_abs = 1.f;         // max |coordinate| over nodes (>= 1)
  // candidate lists: for each node g its K nearest other nodes sorted by the
  // binary32 squared distance w32 = sum (x32 - g32)^2; every node missing from
  // g's list has w32 >= kcert[g]
  int K = 0;
  const int32_t* knn = nullptr;   // [N][K]
  const int32_t* kcnt = nullptr;  // [N] entries in use
  const float* kcert = nullptr;   // [N]
  const float* X32 = nullptr;     // [N][d] nearest binary32 of X, id order
  const float4* X32v = nullptr;   // d <= 8: [N][x32q] the same, rows zero padded to 16-byte vectors
  int x32q = 0;
  double box_lo[16] = {};         // bounding box of all nodes (host copy, binary64)
  double box_hi[16] = {};
  float root_lo[16] = {};         // bounding box of all nodes (binary32, outward)
  float root_hi[16] = {};
};

// Where the rays of a generic raycast come from.
struct RaySource {
  int mode = 0;                  // 0: explicit arrays, 1: MC (cell, ray) list
  int64_t R = 0;
  // explicit
  const double* origins = nullptr;  // R x d
  const double* dirs = nullptr;     // R x d
  const int32_t* eta = nullptr;     // R x eta_stride
  int eta_stride = 0;
  // MC list: ray r is (cell = mc_cell[r], k = mc_ray[r]) of set `set`; with
  // mc_cell == nullptr ray r is (r / mc_rpc, r % mc_rpc)
  const int32_t* mc_cell = nullptr;
  const int32_t* mc_ray = nullptr;
  int64_t mc_rpc = 0;
  uint64_t seed = 0;
  uint32_t set = 0;
  int box = 1;
  int rpb = 32;                  // rays per warp batch (1..32), set by the launcher
  // the ray's output t already holds an upper bound of its hit distance (left
  // there by the list scan that could not certify the ray): start from it
  int t_hint = 0;
  // with R_dev set, the ray count is min(*R_dev, R), read on the device (the
  // launch needs no host round trip), and the batch size is chosen there
  const unsigned long long* R_dev = nullptr;
  // bound on the polls of a device-side wait (tensor-core kernels); 0 = default
  long long wait_limit = 0;
};

struct RayOut {
  int32_t* hit = nullptr;   // R (MC list: indexed cell * mc_rpc + ray)
  double* t = nullptr;      // R
  int64_t mc_rpc = 0;       // rays per cell of the MC output layout
  float* screen_err = nullptr;  // nullable
  int32_t* overflow_list = nullptr;  // rays whose candidate list overflowed
  int64_t overflow_cap = 0;
  int32_t* fallback_list = nullptr;  // rays the candidate lists could not certify
  int64_t fallback_cap = 0;
  double* u = nullptr;  // MC cell kernels: each ray's binary64 direction (row cell * mc_rpc + ray, d values)
  // scratch of the tensor-core list RayCast, which groups the rays by their
  // reference node (grp_ray_ints(N, R) int32 values; null: no grouping)
  int32_t* grp_buf = nullptr;
  int64_t grp_ints = 0;
};

// int32 values of RayOut::grp_buf for N nodes and at most R rays.
int64_t grp_ray_ints(int64_t N, int64_t R);

struct Counters {
  unsigned long long tiles;
  unsigned long long pairs;
  unsigned long long rechecked;
  unsigned long long overflow;
  unsigned long long ties;
  unsigned long long fallback;
  unsigned long long aux0;
  unsigned long long aux1;
  unsigned int flags;
  unsigned int pad;
};

// Polls of a bounded device-side wait for the configured wait_limit: 0 is
// the default (2^22 polls), a negative value gives up before the first poll
// (which tests the time-out path on purpose).
inline long long wait_polls(long long cfg) { return cfg == 0 ? (1ll << 22) : (cfg < 0 ? 0 : cfg); }

// Process-wide count of kernel launches issued by libvd (diagnostics).
extern std::atomic<long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Device allocations owned by one library object, released together.
// Bump allocator over one preallocated device block: many small buffers
// without a cudaMalloc each (and without cudaFree, which synchronises).
struct Arena {
  char* base = nullptr;
  size_t cap = 0, off = 0;
  void* take(size_t bytes) {
    const size_t b = (bytes + 255) / 256 * 256;
    if (!base || off + b > cap) return nullptr;
    void* p = base + off;
    off += b;
    return p;
  }
};

// Device blocks of freed results kept for the next results of the same
// context (result objects share it with the context; the last owner frees
// it): a result of an unchanged size then makes no cudaMalloc or cudaFree.
// Sizes are rounded up to 2 MiB; a block serves a request of at least half
// its size; at most 16 GiB are kept.
struct BufCache {
  std::mutex m;
  std::multimap<size_t, void*> blocks;
  size_t bytes = 0;
  static size_t round(size_t b) { return (b + ((size_t)2 << 20) - 1) / ((size_t)2 << 20) * ((size_t)2 << 20); }
  void* take(size_t b, size_t* got) {
    std::lock_guard<std::mutex> lk(m);
    auto it = blocks.lower_bound(b);
    if (it == blocks.end() || it->first > 2 * b) return nullptr;
    void* p = it->second;
    *got = it->first;
    bytes -= it->first;
    blocks.erase(it);
    return p;
  }
  void give(void* p, size_t b) {
    {
      std::lock_guard<std::mutex> lk(m);
      if (bytes + b <= ((size_t)16 << 30)) {
        blocks.emplace(b, p);
        bytes += b;
        return;
      }
    }
    cudaFree(p);
  }
  ~BufCache() {
    for (auto& kv : blocks) cudaFree(kv.second);
  }
};

struct DevBufs {
  std::vector<void*> ptrs;
  Arena* arena = nullptr;  // if set, buffers come from it while it has room
  size_t requested = 0;    // bytes asked for since the last release (rounded as the arena rounds)
  std::shared_ptr<BufCache> cache;  // if set, blocks come from it and return to it
  std::vector<size_t> sizes;        // with a cache: the block size of each of ptrs
  cudaError_t alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    requested += (bytes + 255) / 256 * 256;
    if (arena && (*p = arena->take(bytes)) != nullptr) return cudaSuccess;
    if (cache) {
      const size_t b = BufCache::round(bytes);
      size_t got = 0;
      if ((*p = cache->take(b, &got)) == nullptr) {
        cudaError_t e = cudaMalloc(p, b);
        if (e != cudaSuccess) return e;
        got = b;
      }
      ptrs.push_back(*p);
      sizes.push_back(got);
      return cudaSuccess;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  template <class T>
  cudaError_t alloc_n(T** p, size_t n) { return alloc(reinterpret_cast<void**>(p), n * sizeof(T)); }
  void release() {
    for (size_t k = 0; k < ptrs.size(); ++k) {
      if (cache && k < sizes.size()) cache->give(ptrs[k], sizes[k]);
      else cudaFree(ptrs[k]);
    }
    ptrs.clear();
    sizes.clear();
    requested = 0;
  }
};

// Device buffers kept across calls: slot k holds one buffer that is
// reallocated only when a call needs more than it holds, so repeated calls of
// the same size make no cudaMalloc / cudaFree (which synchronise the device).
struct Workspace {
  std::vector<std::pair<void*, size_t>> slots;
  cudaError_t get(int slot, size_t bytes, void** p) {
    if (bytes == 0) bytes = 16;
    if ((int)slots.size() <= slot) slots.resize(slot + 1, {nullptr, 0});
    auto& s = slots[slot];
    if (s.second < bytes) {
      if (s.first) cudaFree(s.first);
      s = {nullptr, 0};
      cudaError_t e = cudaMalloc(&s.first, bytes);
      if (e != cudaSuccess) return e;
      s.second = bytes;
    }
    *p = s.first;
    return cudaSuccess;
  }
  template <class T>
  cudaError_t get_n(int slot, size_t n, T** p) {
    return get(slot, n * sizeof(T), reinterpret_cast<void**>(p));
  }
  // 16 words of pinned host memory mapped into the device address space: a
  // kernel writes counters there and the host reads them after a stream
  // synchronisation, with no copy launched
  unsigned long long* host_words = nullptr;
  cudaError_t host_words_get(unsigned long long** p) {
    if (!host_words) {
      cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&host_words), 16 * sizeof(unsigned long long),
                                    cudaHostAllocMapped);
      if (e != cudaSuccess) {
        host_words = nullptr;
        return e;
      }
    }
    *p = host_words;
    return cudaSuccess;
  }
  void release() {
    for (auto& s : slots)
      if (s.first) cudaFree(s.first);
    slots.clear();
    if (host_words) cudaFreeHost(host_words);
    host_words = nullptr;
  }
};

// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum, the same value on every call, so that launches of the same kernel
// with different sizes from several host threads cannot lower the limit
// between another thread's setting and its launch.
template <class Kernel>
inline cudaError_t allow_max_dyn_smem(Kernel kernel) {
  int dev = 0, mx = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess)  // the limit counts the dynamic part only; static shared memory takes the rest
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) cudaGetLastError();  // a later launch check must not see this error
  return e;
}

// ---- launchers (defined in the .cu files) --------------------------------
// Builds the tree of X_dev (N x d, device) into buffers owned by `bufs`.
cudaError_t build_tree(const double* X_dev, int64_t N, int d, cudaStream_t st, DevBufs& bufs, TreeView* tv);
// Builds the per-node candidate lists (K nearest, sorted) into tv.
cudaError_t build_knn(TreeView* tv, int K, cudaStream_t st, DevBufs& bufs);
// Default list length for dimension d (0: no lists, tree walk only).
int default_knn_k(int d);
cudaError_t launch_raycast(const TreeView& tv, const RaySource& rs, const RayOut& ro, int precision,
                           Counters* ctr, cudaStream_t st, int64_t* nfallback = nullptr);
// Same result with no host synchronisation: the ray count may live on the
// device (rs.R_dev, at most rs.R), and the tree-walk and binary64 follow-up
// launches read their counts (ctr->fallback, ctr->overflow) on the device.
// The caller zeroes ctr->fallback and ctr->overflow before the call.
cudaError_t launch_raycast_async(const TreeView& tv, const RaySource& rs, const RayOut& ro, int precision,
                                 Counters* ctr, cudaStream_t st);
// The list scan of explicit rays (rs.mode 0) on the tensor cores: rays
// grouped by reference node, one MMA per chunk of 128 list entries against
// the group's [u; p] rows.  Same contract as the list scan inside
// launch_raycast_async (uncertified rays go to ro.fallback_list, rays whose
// candidate buffer overflows to ro.overflow_list); needs tv.K > 0, d <= 8
// and ro.grp_buf.
cudaError_t launch_list_tc(const TreeView& tv, const RaySource& rs, const RayOut& ro, Counters* ctr,
                           cudaStream_t st);
// Largest coordinate magnitude of a node set the tensor-core kernels take
// (their fp16 operands are offsets of at most twice it).
constexpr float kTcCoordMax = 1.0e4f;
// True when launch_list_tc serves these rays.
inline bool list_tc_ok(const TreeView& tv, const RaySource& rs, const RayOut& ro, int precision) {
  return precision == VD_TC16 && rs.mode == 0 && tv.K > 0 && tv.d <= 8 && tv.coord_abs <= kTcCoordMax &&
         ro.fallback_list != nullptr && ro.grp_buf != nullptr && ro.grp_ints >= grp_ray_ints(tv.N, rs.R);
}
// One point set of a batched MC launch (device array, one entry per set).
struct SetDesc {
  TreeView tv;          // nodes, tiles, candidate lists of the set
  int64_t item0 = 0;    // first global cell index of the set
  uint32_t set = 0;     // Philox set id
  int32_t* hit = nullptr;  // N*R
  double* l = nullptr;     // N*R
  double* V = nullptr;     // N
  int64_t* cnt = nullptr;  // N distinct hits per cell
  int64_t* rowptr = nullptr;  // N+1
  int32_t* col = nullptr;
  double* A = nullptr;
  double cV = 0.0, cA = 0.0;
  Counters* ctr = nullptr;     // per-set counters (fallback, overflow, work)
  int32_t* fb_cell = nullptr;  // rays the lists cannot certify: (cell, ray)
  int32_t* fb_ray = nullptr;
  int64_t fb_cap = 0;
  int32_t* ov_list = nullptr;  // rays the binary32 screen could not settle
  int64_t ov_cap = 0;
};

// Batched forward pass over nsets sets (items = all cells of all sets), no
// host synchronisation: cell kernel (brute-force binary64 finish for rays
// the lists cannot certify), distinct-hit counts, per-set scans, fill.
cudaError_t launch_mc_batch(const SetDesc* sets_dev, const SetDesc* sets_host, int nsets, int64_t nitems, int maxd,
                            int maxK, int64_t R, uint64_t seed, int threads, Counters* ctr, cudaStream_t st);
cudaError_t launch_mc_batch_cells(const SetDesc* sets_dev, const SetDesc* sets_host, int nsets, int64_t nitems,
                                  int maxK, int64_t R, uint64_t seed, int threads, Counters* ctr, cudaStream_t st);
// Tree-walk finish of one set's uncertified MC rays with device-side counts.
cudaError_t launch_mc_fallback_dev(const SetDesc& S, int64_t R, uint64_t seed, cudaStream_t st);
void mc_batch_dims(int threads, int maxd, int maxK, size_t* smem);

// MC rays of all cells through the cell-centric kernel (candidate lists
// required), leftovers through launch_raycast.  ro.fallback_list holds
// 2 x (fallback_cap / 2) entries for (cell, ray) pairs.
cudaError_t launch_mc_cells(const TreeView& tv, int64_t R, uint64_t seed, uint32_t set, const RayOut& ro,
                            int precision, Counters* ctr, cudaStream_t st, int64_t* nfallback);
// Same contract with the u.w screening contraction on the tensor cores
// (tcgen05, fp16 operands); needs coordinates within the fp16 range
// (tv.coord_abs <= kTcCoordMax).  MMA completion waits poll at most
// wait_limit times; a wait that gives up sets kFlagTimeout.
cudaError_t launch_mc_cells_tc(const TreeView& tv, int64_t R, uint64_t seed, uint32_t set, const RayOut& ro,
                               Counters* ctr, long long wait_limit, cudaStream_t st, int64_t* nfallback);
// MC rays without candidate lists: block tree walk with the ball tests of
// children and the leaf screening on the tensor cores; same contract as
// launch_mc_cells_tc.
cudaError_t launch_mc_walk_tc(const TreeView& tv, int64_t R, uint64_t seed, uint32_t set, const RayOut& ro,
                              Counters* ctr, long long wait_limit, cudaStream_t st, int64_t* nfallback);
cudaError_t launch_mc_directions(uint64_t seed, uint32_t set, int64_t cell0, int64_t ncells, int64_t R, int d,
                                 double* out, cudaStream_t st);

}  // namespace vd
