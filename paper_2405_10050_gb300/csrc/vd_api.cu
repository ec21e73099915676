// vd_api.cu -- the extern "C" entry points of libvd (include/vd.h): argument
// checks, host/device staging, object lifetimes and launch sequencing.  All
// arithmetic of the method runs in the kernels of the other files.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "vd_dev.cuh"

namespace vd {
cudaError_t mc_rowptr(const int32_t* hit, int64_t N, int64_t R, int64_t* cnt_scratch, int64_t* rowptr,
                      int64_t* nnz_host, cudaStream_t st);
cudaError_t mc_fill(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set, const int32_t* hit,
                    const double* l, const int64_t* rowptr, double* V, int32_t* col, double* A, const double* U,
                    cudaStream_t st);
cudaError_t mc_adjoint(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set,
                       const int32_t* hit, const double* l, const int64_t* rowptr, const int32_t* col, int64_t nnz,
                       const double* gV, const double* gA, double* gX, const double* U, DevBufs& scratch,
                       cudaStream_t st);
cudaError_t mc_integrals(const double* X, int64_t N, int d, int64_t R, uint64_t seed, uint32_t set,
                         const int32_t* hit, const double* l, const int64_t* rowptr, const int32_t* col,
                         const double* U, const vd_func& f, int64_t m, double* FV, double* Fd, cudaStream_t st);
cudaError_t hmc_integrals(const double* X, int64_t N, int d, const int64_t* rowptr, const int32_t* col,
                          const double* A, int64_t nnz, const int32_t* tuples, const double* coords, int64_t nv,
                          const vd_func& f, double* VH, double* FH, double* IH, DevBufs& scratch, cudaStream_t st);
cudaError_t poly_integrate(const double* X, int64_t N, int d, const int32_t* tuples, const double* coords,
                           int64_t nv, const vd_func& f, DevBufs& out, DevBufs& scratch, double** V, double** F,
                           int64_t** rowptr, int32_t** col, double** A, double** Fd, int64_t* nnz, unsigned* flags_h,
                           cudaStream_t st);
cudaError_t random_walk(const TreeView& tv, int precision, const int32_t* start, int64_t W, int64_t S, uint64_t seed,
                        int32_t* path_t, double* path_x, Counters* ctr, DevBufs& scratch, cudaStream_t st,
                        double* raycast_ms);
cudaError_t traverse_vertices(const TreeView& tv, int precision, const vd_config& cfg, int64_t cells_per_batch,
                              Workspace& ws, DevBufs& out_bufs, int32_t** tuples, double** coords, int64_t* nv,
                              vd_stats* stats, Counters* ctr, cudaStream_t st, char* err, size_t errlen);
}  // namespace vd

namespace vd {
std::atomic<long long> g_launches{0};
}

using vd::Counters;
using vd::DevBufs;
using vd::TreeView;

struct vd_ctx {
  vd_config cfg;
  int dev = -1;  // the CUDA device current at vd_create
  cudaStream_t st = nullptr;
  char err[512] = {0};
  vd_stats last{};
  DevBufs node_bufs;
  // one device block that the node set's buffers are carved from (sized by
  // the previous node set), so that setting nodes of an unchanged size makes
  // no cudaMalloc or cudaFree (both synchronise the device)
  vd::Arena node_arena;
  // device blocks of freed MC results and meshes, for the next ones
  std::shared_ptr<vd::BufCache> result_cache = std::make_shared<vd::BufCache>();
  TreeView tree;
  double* X = nullptr;
  int64_t N = 0;
  int d = 0;
  Counters* ctr = nullptr;  // device
  DevBufs own;
  int batch_threads[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // autotuned block size by largest d
  vd::Workspace trav_ws;  // traversal tables and level buffers, reused across vd_vertices calls
  vd::Workspace mc_ws;    // MC work lists, reused across vd_mc_integrate calls
  vd::Workspace batch_ws; // batched MC: trees, candidate lists, work lists of all sets (one block)
  // batched MC forward pass: the instantiated graph, updated in place by the
  // next call's capture (instantiated again only when its shape changes)
  cudaGraphExec_t batch_exec = nullptr;
};

struct vd_mesh {
  cudaStream_t st = nullptr;
  int d = 0;
  int64_t nv = 0;
  DevBufs bufs;
  int32_t* tuples = nullptr;  // device, sorted rows, lexicographic order
  double* coords = nullptr;
  vd_stats stats{};
};

struct vd_mc {
  cudaStream_t st = nullptr;
  int64_t N = 0, R = 0, nnz = 0;
  int d = 0;
  uint64_t seed = 0;
  uint32_t set = 0;
  DevBufs bufs;
  double* X = nullptr;
  int32_t* hit = nullptr;
  double* l = nullptr;
  double* u = nullptr;  // ray directions kept from the forward pass (or null: drawn again)
  std::shared_ptr<void> pool;  // batched sets: one device block shared by all of a batch's results
  double* V = nullptr;
  int64_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* A = nullptr;
  vd_stats stats{};
};

struct vd_poly {
  cudaStream_t st = nullptr;
  int64_t N = 0, nnz = 0;
  DevBufs bufs;
  double *V = nullptr, *F = nullptr, *A = nullptr, *Fd = nullptr;
  int64_t* rowptr = nullptr;
  int32_t* col = nullptr;
};

namespace {

vd_status set_err(vd_ctx* c, vd_status s, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

vd_status cuda_err(vd_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return set_err(c, VD_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
  return set_err(c, VD_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define VD_CK(call, where)                                \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, where); \
  } while (0)

// Stages an input array on the device (copy for host memory).
template <class T>
vd_status stage_in(vd_ctx* ctx, DevBufs& tmp, const T* src, size_t n, int on_device, const T** out) {
  if (on_device || n == 0) {
    *out = src;
    return VD_OK;
  }
  T* p = nullptr;
  VD_CK(tmp.alloc_n(&p, n), "stage_in alloc");
  VD_CK(cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyHostToDevice, ctx->st), "stage_in copy");
  *out = p;
  return VD_OK;
}

struct Timer {
  cudaEvent_t a{}, b{};
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

vd_status read_counters(vd_ctx* ctx, Counters* hc) {
  VD_CK(cudaMemcpyAsync(hc, ctx->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->st), "counters");
  VD_CK(cudaStreamSynchronize(ctx->st), "sync");
  return VD_OK;
}

vd_status check_flags(vd_ctx* ctx, const Counters& hc) {
  if (hc.flags & vd::kFlagBadInput)
    return set_err(ctx, VD_EINVAL, "a ray's first eta entry (its reference generator g) is not a node id");
  if (hc.flags & vd::kFlagHashFull) return set_err(ctx, VD_EHASHFULL, "device table capacity reached");
  if (hc.flags & vd::kFlagTimeout) return set_err(ctx, VD_ETIMEOUT, "bounded device wait gave up");
  if (hc.flags & (vd::kFlagCandOverflow | vd::kFlagQueue | vd::kFlagStack))
    return set_err(ctx, VD_EOVERFLOW, "device work list overflow (flags 0x%x)", hc.flags);
  if (hc.flags & vd::kFlagDegenerate) return set_err(ctx, VD_EDEGENERATE, "degenerate configuration");
  return VD_OK;
}

// The path of a call.  VD_AUTO takes the fastest path measured on GB300 for
// the call's kind and node set:
//  * Monte Carlo rays: the tensor-core block walk for node sets without
//    candidate lists (d > 8; d = 16, N = 200,000: ten times the binary32
//    tree walk), else the binary32 cell kernel (d = 4: 1.43M against 1.19M
//    cells/s on the tensor-core cells);
//  * explicit rays (vd_raycast, vd_vertices, vd_random_walk) with candidate
//    lists: the tensor-core list scan for 3 <= d <= 8 (traversal raycasts/s
//    5-25 % above binary32 at d = 3..6), binary32 at d <= 2.
int effective_precision(const vd_ctx* ctx, bool mc = false) {
  const int p = ctx->cfg.precision;
  if (p == VD_FP64 || p == VD_FP32 || p == VD_TC16) return p;
  const vd::TreeView& tv = ctx->tree;
  const bool tc_range = tv.coord_abs <= vd::kTcCoordMax;
  if (mc) return (tv.K == 0 && tc_range) ? VD_TC16 : VD_FP32;
  return (tv.K > 0 && tv.d >= 3 && tv.d <= 8 && tc_range) ? VD_TC16 : VD_FP32;
}

}  // namespace

extern "C" {

int64_t vd_kernel_launches(void) { return (int64_t)vd::g_launches.load(); }

void vd_config_default(vd_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->precision = VD_AUTO;
  cfg->box = 1;
  cfg->wait_limit = 1 << 22;
}

const char* vd_status_str(vd_status s) {
  switch (s) {
    case VD_OK: return "ok";
    case VD_EINVAL: return "invalid argument";
    case VD_ENOMEM: return "out of memory";
    case VD_ECUDA: return "CUDA error";
    case VD_EDEGENERATE: return "degenerate input";
    case VD_EHASHFULL: return "hash table full";
    case VD_EOVERFLOW: return "work list overflow";
    case VD_ETIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

vd_status vd_create(vd_ctx** out, const vd_config* cfg, void* stream) {
  if (!out) return VD_EINVAL;
  *out = nullptr;
  vd_ctx* ctx = new (std::nothrow) vd_ctx();
  if (!ctx) return VD_ENOMEM;
  if (cfg) ctx->cfg = *cfg;
  else vd_config_default(&ctx->cfg);
  if (ctx->cfg.precision < VD_FP64 || ctx->cfg.precision > VD_AUTO) {
    delete ctx;
    return VD_EINVAL;
  }
  ctx->st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&ctx->dev);
  if (e == cudaSuccess) e = ctx->own.alloc_n(&ctx->ctr, 1);
  if (e != cudaSuccess) {
    delete ctx;
    return e == cudaErrorMemoryAllocation ? VD_ENOMEM : VD_ECUDA;
  }
  *out = ctx;
  return VD_OK;
}

void vd_destroy(vd_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->st);
  ctx->node_bufs.release();
  if (ctx->node_arena.base) cudaFree(ctx->node_arena.base);
  ctx->own.release();
  ctx->trav_ws.release();
  ctx->mc_ws.release();
  ctx->batch_ws.release();
  if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
  delete ctx;
}

const char* vd_last_error(const vd_ctx* ctx) { return ctx ? ctx->err : "null context"; }

vd_status vd_set_precision(vd_ctx* ctx, int32_t precision) {
  if (!ctx || precision < VD_FP64 || precision > VD_AUTO) return VD_EINVAL;
  ctx->cfg.precision = precision;
  return VD_OK;
}

vd_status vd_last_stats(const vd_ctx* ctx, vd_stats* out) {
  if (!ctx || !out) return VD_EINVAL;
  *out = ctx->last;
  return VD_OK;
}

vd_status vd_set_nodes(vd_ctx* ctx, const double* X, int64_t N, int32_t d, int32_t on_device) {
  if (!ctx) return VD_EINVAL;
  if (!X || N < 1 || d < 1 || d > VD_MAX_D || N > (int64_t)1 << 30)
    return set_err(ctx, VD_EINVAL, "vd_set_nodes: need X, 1 <= N <= 2^30, 1 <= d <= 16 (N=%lld d=%d)",
                   (long long)N, d);
  VD_CK(cudaStreamSynchronize(ctx->st), "sync");
  // the previous set asked for `requested` bytes: keep a block that holds them
  const size_t need = ctx->node_bufs.requested;
  ctx->node_bufs.release();
  if (need > ctx->node_arena.cap) {
    if (ctx->node_arena.base) cudaFree(ctx->node_arena.base);
    ctx->node_arena.base = nullptr;
    ctx->node_arena.cap = 0;
    const size_t cap = need + need / 8;
    if (cudaMalloc(reinterpret_cast<void**>(&ctx->node_arena.base), cap) == cudaSuccess) ctx->node_arena.cap = cap;
    else cudaGetLastError();
  }
  ctx->node_arena.off = 0;
  ctx->node_bufs.arena = &ctx->node_arena;
  ctx->X = nullptr;
  ctx->N = 0;
  ctx->d = 0;
  double* Xd = nullptr;
  VD_CK(ctx->node_bufs.alloc_n(&Xd, (size_t)N * d), "nodes alloc");
  VD_CK(cudaMemcpyAsync(Xd, X, (size_t)N * d * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->st),
        "nodes copy");
  TreeView tv;
  cudaError_t e = vd::build_tree(Xd, N, d, ctx->st, ctx->node_bufs, &tv);
  if (e == cudaErrorInvalidValue) {
    ctx->node_bufs.release();
    return set_err(ctx, VD_EINVAL, "vd_set_nodes: non-finite coordinate");
  }
  if (e != cudaSuccess) {
    ctx->node_bufs.release();
    return cuda_err(ctx, e, "build_tree");
  }
  const int K = ctx->cfg.knn_k < 0 ? 0 : (ctx->cfg.knn_k > 0 ? ctx->cfg.knn_k : vd::default_knn_k(d));
  if (K > 0 && d <= 8) {
    const int Kuse = (int)std::min<int64_t>(K, std::max<int64_t>(N - 1, 1));
    e = vd::build_knn(&tv, Kuse, ctx->st, ctx->node_bufs);
    if (e != cudaSuccess) {
      ctx->node_bufs.release();
      return cuda_err(ctx, e, "build_knn");
    }
  }
  ctx->tree = tv;
  ctx->X = Xd;
  ctx->N = N;
  ctx->d = d;
  return VD_OK;
}

vd_status vd_raycast(vd_ctx* ctx, const double* origins, const double* dirs, const int32_t* eta, int32_t eta_stride,
                     int64_t R, int32_t* hit, double* t, float* screen_err, int32_t on_device) {
  if (!ctx) return VD_EINVAL;
  if (!ctx->X) return set_err(ctx, VD_EINVAL, "vd_raycast: no node set");
  if (R < 0 || (R > 0 && (!origins || !dirs || !eta || !hit || !t)) || eta_stride < 1 ||
      eta_stride > ctx->d + 1)
    return set_err(ctx, VD_EINVAL, "vd_raycast: bad arguments (R=%lld, eta_stride=%d, d=%d)", (long long)R,
                   eta_stride, ctx->d);
  ctx->last = vd_stats{};
  if (R == 0) return VD_OK;
  const int d = ctx->d;
  DevBufs tmp;
  struct Guard {
    DevBufs& b;
    ~Guard() { b.release(); }
  } guard{tmp};
  const double *o_d, *u_d;
  const int32_t* e_d;
  vd_status s;
  if ((s = stage_in(ctx, tmp, origins, (size_t)R * d, on_device, &o_d)) != VD_OK) return s;
  if ((s = stage_in(ctx, tmp, dirs, (size_t)R * d, on_device, &u_d)) != VD_OK) return s;
  if ((s = stage_in(ctx, tmp, eta, (size_t)R * eta_stride, on_device, &e_d)) != VD_OK) return s;
  int32_t* h_d = hit;
  double* t_d = t;
  float* se_d = screen_err;
  if (!on_device) {
    VD_CK(tmp.alloc_n(&h_d, R), "alloc");
    VD_CK(tmp.alloc_n(&t_d, R), "alloc");
    if (screen_err) VD_CK(tmp.alloc_n(&se_d, R), "alloc");
  }
  int32_t *ovl = nullptr, *fbl = nullptr;
  const int64_t ovcap = R;  // every ray may overflow its binary32 candidate buffer (clustered nodes)
  VD_CK(tmp.alloc_n(&ovl, ovcap), "alloc");
  VD_CK(tmp.alloc_n(&fbl, R), "alloc");
  int32_t* grp = nullptr;
  const int64_t grp_ints = effective_precision(ctx) == VD_TC16 ? vd::grp_ray_ints(ctx->N, R) : 0;
  if (grp_ints > 0) VD_CK(tmp.alloc_n(&grp, (size_t)grp_ints), "alloc");
  // eta rows must start with a node
  vd::RaySource rs;
  rs.mode = 0;
  rs.R = R;
  rs.origins = o_d;
  rs.dirs = u_d;
  rs.eta = e_d;
  rs.eta_stride = eta_stride;
  rs.box = ctx->cfg.box;
  vd::RayOut ro;
  ro.hit = h_d;
  ro.t = t_d;
  ro.screen_err = se_d;
  ro.overflow_list = ovl;
  ro.overflow_cap = ovcap;
  ro.fallback_list = fbl;
  ro.fallback_cap = R;
  ro.grp_buf = grp;
  ro.grp_ints = grp_ints;
  rs.wait_limit = ctx->cfg.wait_limit;
  VD_CK(cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), ctx->st), "memset");
  const long long l0 = vd::g_launches.load();
  Timer tm(ctx->st);
  int64_t nfb = 0;
  VD_CK(vd::launch_raycast(ctx->tree, rs, ro, effective_precision(ctx), ctx->ctr, ctx->st, &nfb), "raycast");
  ctx->last.fallback_rays = nfb;
  ctx->last.ms = tm.stop();
  ctx->last.raycast_ms = ctx->last.ms;
  ctx->last.launches = vd::g_launches.load() - l0;
  if (!on_device) {
    VD_CK(cudaMemcpyAsync(hit, h_d, R * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st), "copy out");
    VD_CK(cudaMemcpyAsync(t, t_d, R * sizeof(double), cudaMemcpyDeviceToHost, ctx->st), "copy out");
    if (screen_err) VD_CK(cudaMemcpyAsync(screen_err, se_d, R * sizeof(float), cudaMemcpyDeviceToHost, ctx->st), "copy out");
  }
  Counters hc;
  if ((s = read_counters(ctx, &hc)) != VD_OK) return s;
  ctx->last.rays = R;
  ctx->last.tiles_visited = (int64_t)hc.tiles;
  ctx->last.pairs_screened = (int64_t)hc.pairs;
  ctx->last.rechecked = (int64_t)hc.rechecked;
  ctx->last.overflow_rays = (int64_t)hc.overflow;
  return check_flags(ctx, hc);
}

vd_status vd_mc_directions(vd_ctx* ctx, uint64_t seed, uint32_t set, int64_t cell0, int64_t ncells, int64_t R,
                           int32_t d, double* out, int32_t on_device) {
  if (!ctx) return VD_EINVAL;
  if (!out || cell0 < 0 || ncells < 0 || R < 0 || d < 1 || d > VD_MAX_D || cell0 + ncells > ((int64_t)1 << 32) ||
      R > ((int64_t)1 << 32))
    return set_err(ctx, VD_EINVAL, "vd_mc_directions: bad arguments");
  const int64_t n = ncells * R * d;
  if (n == 0) return VD_OK;
  DevBufs tmp;
  double* o = out;
  if (!on_device) VD_CK(tmp.alloc_n(&o, n), "alloc");
  cudaError_t e = vd::launch_mc_directions(seed, set, cell0, ncells, R, d, o, ctx->st);
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, o, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  tmp.release();
  if (e != cudaSuccess) return cuda_err(ctx, e, "mc_directions");
  return VD_OK;
}

// ---------------------------------------------------------------- MC ----
static vd_status mc_run(vd_ctx* ctx, const TreeView& tv, double* Xd, int64_t N, int d, int64_t R, uint64_t seed,
                        uint32_t set, vd_mc* mc) {
  mc->st = ctx->st;
  mc->N = N;
  mc->d = d;
  mc->R = R;
  mc->seed = seed;
  mc->set = set;
  mc->X = Xd;
  VD_CK(mc->bufs.alloc_n(&mc->hit, (size_t)N * R), "mc alloc");
  VD_CK(mc->bufs.alloc_n(&mc->l, (size_t)N * R), "mc alloc");
  VD_CK(mc->bufs.alloc_n(&mc->V, (size_t)N), "mc alloc");
  VD_CK(mc->bufs.alloc_n(&mc->rowptr, (size_t)N + 1), "mc alloc");
  int32_t *ovl = nullptr, *fbl = nullptr;
  int64_t* cnt = nullptr;
  const int64_t ovcap = std::max<int64_t>(4096, N * R / 64);
  VD_CK(ctx->mc_ws.get_n(0, ovcap, &ovl), "alloc");
  VD_CK(ctx->mc_ws.get_n(1, N * R, &fbl), "alloc");
  VD_CK(ctx->mc_ws.get_n(2, N, &cnt), "alloc");
  const int prec = effective_precision(ctx, true);
  // the cell kernels keep each ray's binary64 direction for the fill and the
  // adjoint (8 d bytes per ray) unless that would exceed 16 GiB
  const bool cells = tv.K > 0;
  if (cells && (double)N * R * d * 8.0 <= 16.0 * (1ull << 30))
    VD_CK(mc->bufs.alloc_n(&mc->u, (size_t)N * R * d), "mc alloc");
  vd::RaySource rs;
  rs.mode = 1;
  rs.R = N * R;
  rs.mc_rpc = R;
  rs.seed = seed;
  rs.set = set;
  rs.box = 1;
  vd::RayOut ro;
  ro.hit = mc->hit;
  ro.t = mc->l;
  ro.mc_rpc = R;
  ro.overflow_list = ovl;
  ro.overflow_cap = ovcap;
  ro.fallback_list = fbl;
  ro.fallback_cap = N * R;
  ro.u = mc->u;
  VD_CK(cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), ctx->st), "memset");
  const long long l0 = vd::g_launches.load();
  Timer tm(ctx->st);
  {
    Timer tr(ctx->st);
    if (tv.K > 0 && prec == VD_TC16 && tv.coord_abs <= vd::kTcCoordMax)
      VD_CK(vd::launch_mc_cells_tc(tv, R, seed, set, ro, ctx->ctr, ctx->cfg.wait_limit, ctx->st,
                                   &mc->stats.fallback_rays),
            "mc cells tc");
    else if (prec == VD_TC16 && tv.coord_abs <= vd::kTcCoordMax)
      VD_CK(vd::launch_mc_walk_tc(tv, R, seed, set, ro, ctx->ctr, ctx->cfg.wait_limit, ctx->st,
                                  &mc->stats.fallback_rays),
            "mc walk tc");
    else if (tv.K > 0)  // binary32 screening, or every pair in binary64 (same list scan)
      VD_CK(vd::launch_mc_cells(tv, R, seed, set, ro, prec, ctx->ctr, ctx->st, &mc->stats.fallback_rays),
            "mc cells");
    else
      VD_CK(vd::launch_raycast(tv, rs, ro, prec, ctx->ctr, ctx->st, &mc->stats.fallback_rays), "mc raycast");
    mc->stats.raycast_ms = tr.stop();
  }
  {
    // a tensor-core kernel that gave up a bounded wait left rays without a
    // hit: stop before the kernels that read the hits
    Counters hc0;
    vd_status s0 = read_counters(ctx, &hc0);
    if (s0 != VD_OK) return s0;
    if (hc0.flags & vd::kFlagTimeout) return check_flags(ctx, hc0);
  }
  int64_t nnz = 0;
  VD_CK(vd::mc_rowptr(mc->hit, N, R, cnt, mc->rowptr, &nnz, ctx->st), "mc rowptr");
  mc->nnz = nnz;
  VD_CK(mc->bufs.alloc_n(&mc->col, (size_t)std::max<int64_t>(nnz, 1)), "mc alloc");
  VD_CK(mc->bufs.alloc_n(&mc->A, (size_t)std::max<int64_t>(nnz, 1)), "mc alloc");
  VD_CK(vd::mc_fill(Xd, N, d, R, seed, set, mc->hit, mc->l, mc->rowptr, mc->V, mc->col, mc->A, mc->u, ctx->st),
        "mc fill");
  mc->stats.ms = tm.stop();
  mc->stats.launches = vd::g_launches.load() - l0;
  Counters hc;
  vd_status s;
  if ((s = read_counters(ctx, &hc)) != VD_OK) return s;
  mc->stats.rays = N * R;
  mc->stats.tiles_visited = (int64_t)hc.tiles;
  mc->stats.pairs_screened = (int64_t)hc.pairs;
  mc->stats.rechecked = (int64_t)hc.rechecked;
  mc->stats.overflow_rays = (int64_t)hc.overflow;
  ctx->last = mc->stats;
  return check_flags(ctx, hc);
}

vd_status vd_mc_integrate(vd_ctx* ctx, int64_t R, uint64_t seed, vd_mc** out) {
  if (!ctx || !out) return VD_EINVAL;
  *out = nullptr;
  if (!ctx->X) return set_err(ctx, VD_EINVAL, "vd_mc_integrate: no node set");
  if (!ctx->cfg.box) return set_err(ctx, VD_EINVAL, "vd_mc_integrate: needs box clipping (cells are unbounded)");
  if (R < 1 || R > ((int64_t)1 << 31) || ctx->N * R > ((int64_t)1 << 40))
    return set_err(ctx, VD_EINVAL, "vd_mc_integrate: bad rays_per_cell %lld", (long long)R);
  vd_mc* mc = new (std::nothrow) vd_mc();
  if (!mc) return VD_ENOMEM;
  mc->bufs.cache = ctx->result_cache;
  double* Xc = nullptr;
  cudaError_t e = mc->bufs.alloc_n(&Xc, (size_t)ctx->N * ctx->d);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Xc, ctx->X, (size_t)ctx->N * ctx->d * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st);
  if (e != cudaSuccess) {
    mc->bufs.release();
    delete mc;
    return cuda_err(ctx, e, "mc alloc");
  }
  vd_status s = mc_run(ctx, ctx->tree, Xc, ctx->N, ctx->d, R, seed, 0, mc);
  if (s != VD_OK) {
    cudaStreamSynchronize(ctx->st);
    mc->bufs.release();
    delete mc;
    return s;
  }
  *out = mc;
  return VD_OK;
}

int64_t vd_mc_count(const vd_mc* mc) { return mc ? mc->N : 0; }

vd_status vd_mc_stats(const vd_mc* mc, vd_stats* out) {
  if (!mc || !out) return VD_EINVAL;
  *out = mc->stats;
  return VD_OK;
}

vd_status vd_mc_get(const vd_mc* mc, double* V, int64_t* nnz, int64_t* rowptr, int32_t* col, double* A,
                    int32_t on_device) {
  if (!mc) return VD_EINVAL;
  if (nnz) *nnz = mc->nnz;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  if (V && e == cudaSuccess) e = cudaMemcpyAsync(V, mc->V, mc->N * sizeof(double), k, mc->st);
  if (rowptr && e == cudaSuccess) e = cudaMemcpyAsync(rowptr, mc->rowptr, (mc->N + 1) * sizeof(int64_t), k, mc->st);
  if (col && e == cudaSuccess && mc->nnz) e = cudaMemcpyAsync(col, mc->col, mc->nnz * sizeof(int32_t), k, mc->st);
  if (A && e == cudaSuccess && mc->nnz) e = cudaMemcpyAsync(A, mc->A, mc->nnz * sizeof(double), k, mc->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mc->st);
  return e == cudaSuccess ? VD_OK : VD_ECUDA;
}

vd_status vd_mc_rays(const vd_mc* mc, int32_t* hit, double* l, int32_t on_device) {
  if (!mc) return VD_EINVAL;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  if (hit) e = cudaMemcpyAsync(hit, mc->hit, mc->N * mc->R * sizeof(int32_t), k, mc->st);
  if (l && e == cudaSuccess) e = cudaMemcpyAsync(l, mc->l, mc->N * mc->R * sizeof(double), k, mc->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mc->st);
  return e == cudaSuccess ? VD_OK : VD_ECUDA;
}

vd_status vd_mc_adjoint(const vd_mc* mc, const double* gV, const double* gA, double* gX, int32_t on_device) {
  if (!mc || !gX || (!gV && !gA)) return VD_EINVAL;
  // scratch of up to 1 GiB comes from a block this thread keeps for its next
  // calls (many small adjoints, e.g. of a batch, then allocate nothing)
  static thread_local vd::Workspace tl_ws;
  const size_t nn = (size_t)std::max<int64_t>(mc->nnz, 1), n = (size_t)mc->N, dd = (size_t)mc->d;
  const size_t need = 256 * 16 + nn * dd * 8 + n * dd * 8 * 2 + nn * 24 + 1024 * (nn / 4096 + 2) + n * 8 * 2 + nn * 8;
  vd::Arena arena;
  if (need <= ((size_t)1 << 30)) {
    void* b = nullptr;
    if (tl_ws.get(0, need, &b) == cudaSuccess) arena = vd::Arena{static_cast<char*>(b), need, 0};
  }
  DevBufs tmp;
  tmp.arena = &arena;
  const double *gVd = gV, *gAd = gA;
  double* gXd = gX;
  double* zeroV = nullptr;
  cudaError_t e = cudaSuccess;
  auto stage = [&](const double* src, size_t n, const double** dst) {
    if (on_device || !src || e != cudaSuccess) return;
    double* p = nullptr;
    e = tmp.alloc_n(&p, n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, src, n * sizeof(double), cudaMemcpyHostToDevice, mc->st);
    *dst = p;
  };
  stage(gV, mc->N, &gVd);
  stage(gA, mc->nnz, &gAd);
  if (e == cudaSuccess && !gVd) {
    e = tmp.alloc_n(&zeroV, mc->N);
    if (e == cudaSuccess) e = cudaMemsetAsync(zeroV, 0, mc->N * sizeof(double), mc->st);
    gVd = zeroV;
  }
  if (e == cudaSuccess && !on_device) e = tmp.alloc_n(&gXd, (size_t)mc->N * mc->d);
  if (e == cudaSuccess)
    e = vd::mc_adjoint(mc->X, mc->N, mc->d, mc->R, mc->seed, mc->set, mc->hit, mc->l, mc->rowptr, mc->col, mc->nnz,
                       gVd, gAd, gXd, mc->u, tmp, mc->st);
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(gX, gXd, (size_t)mc->N * mc->d * sizeof(double), cudaMemcpyDeviceToHost, mc->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mc->st);
  cudaStreamSynchronize(mc->st);
  tmp.release();
  return e == cudaSuccess ? VD_OK : (e == cudaErrorMemoryAllocation ? VD_ENOMEM : VD_ECUDA);
}

static bool func_ok(const vd_func* f, int d) {
  if (f->kind != VD_F_ONE && f->kind != VD_F_POLY2 && f->kind != VD_F_SIN_SQ) return false;
  return f->kind != VD_F_SIN_SQ || (f->axis >= 0 && f->axis < d);
}

vd_status vd_mc_integrals(const vd_mc* mc, const vd_func* f, int64_t m, double* FV, double* Fd, int32_t on_device) {
  if (!mc || !f || (!FV && !Fd)) return VD_EINVAL;
  if (!func_ok(f, mc->d)) return VD_EINVAL;
  if (FV && (m < 1 || m > ((int64_t)1 << 32))) return VD_EINVAL;  // sample blocks s / 4 below 2^31
  if (!FV) m = 1;
  DevBufs tmp;
  double *FVd = FV, *Fdd = Fd;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    if (FV) e = tmp.alloc_n(&FVd, (size_t)mc->N);
    if (e == cudaSuccess && Fd) e = tmp.alloc_n(&Fdd, (size_t)std::max<int64_t>(mc->nnz, 1));
  }
  if (e == cudaSuccess)
    e = vd::mc_integrals(mc->X, mc->N, mc->d, mc->R, mc->seed, mc->set, mc->hit, mc->l, mc->rowptr, mc->col, mc->u, *f,
                         m, FVd, Fdd, mc->st);
  if (e == cudaSuccess && !on_device && FV)
    e = cudaMemcpyAsync(FV, FVd, (size_t)mc->N * sizeof(double), cudaMemcpyDeviceToHost, mc->st);
  if (e == cudaSuccess && !on_device && Fd && mc->nnz > 0)
    e = cudaMemcpyAsync(Fd, Fdd, (size_t)mc->nnz * sizeof(double), cudaMemcpyDeviceToHost, mc->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mc->st);
  cudaStreamSynchronize(mc->st);
  tmp.release();
  return e == cudaSuccess ? VD_OK : (e == cudaErrorMemoryAllocation ? VD_ENOMEM : VD_ECUDA);
}

vd_status vd_hmc_integrals(const vd_mc* mc, const vd_mesh* mesh, const vd_func* f, double* VH, double* FH,
                           double* IH, int32_t on_device) {
  if (!mc || !mesh || !f || (!VH && !FH && !IH)) return VD_EINVAL;
  if (mesh->d != mc->d || !func_ok(f, mc->d)) return VD_EINVAL;
  DevBufs tmp;
  double *VHd = VH, *FHd = FH, *IHd = IH;
  cudaError_t e = cudaSuccess;
  if (VH && !on_device) e = tmp.alloc_n(&VHd, (size_t)mc->N);
  if (e == cudaSuccess && IH && !on_device) e = tmp.alloc_n(&IHd, (size_t)mc->N);
  if (e == cudaSuccess && (!FH || !on_device)) e = tmp.alloc_n(&FHd, (size_t)std::max<int64_t>(mc->nnz, 1));
  if (e == cudaSuccess)
    e = vd::hmc_integrals(mc->X, mc->N, mc->d, mc->rowptr, mc->col, mc->A, mc->nnz, mesh->tuples, mesh->coords,
                          mesh->nv, *f, VHd, FHd, IHd, tmp, mc->st);
  if (e == cudaSuccess && !on_device && VH)
    e = cudaMemcpyAsync(VH, VHd, (size_t)mc->N * sizeof(double), cudaMemcpyDeviceToHost, mc->st);
  if (e == cudaSuccess && !on_device && IH)
    e = cudaMemcpyAsync(IH, IHd, (size_t)mc->N * sizeof(double), cudaMemcpyDeviceToHost, mc->st);
  if (e == cudaSuccess && !on_device && FH && mc->nnz > 0)
    e = cudaMemcpyAsync(FH, FHd, (size_t)mc->nnz * sizeof(double), cudaMemcpyDeviceToHost, mc->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mc->st);
  cudaStreamSynchronize(mc->st);
  tmp.release();
  return e == cudaSuccess ? VD_OK : (e == cudaErrorMemoryAllocation ? VD_ENOMEM : VD_ECUDA);
}

vd_status vd_poly_integrate(vd_ctx* ctx, const vd_mesh* mesh, const vd_func* f, vd_poly** out) {
  if (!ctx || !mesh || !f || !out) return VD_EINVAL;
  *out = nullptr;
  if (!ctx->X) return set_err(ctx, VD_EINVAL, "vd_poly_integrate: no nodes set");
  if (mesh->d != ctx->d || ctx->d < 2 || ctx->d > 8)
    return set_err(ctx, VD_EINVAL, "vd_poly_integrate: needs the mesh of the context's nodes and 2 <= d <= 8");
  if (!func_ok(f, ctx->d)) return set_err(ctx, VD_EINVAL, "vd_poly_integrate: bad function");
  vd_poly* p = new (std::nothrow) vd_poly;
  if (!p) return VD_ENOMEM;
  p->st = ctx->st;
  p->N = ctx->N;
  DevBufs scratch;
  unsigned flags = 0;
  cudaError_t e = vd::poly_integrate(ctx->X, ctx->N, ctx->d, mesh->tuples, mesh->coords, mesh->nv, *f, p->bufs,
                                     scratch, &p->V, &p->F, &p->rowptr, &p->col, &p->A, &p->Fd, &p->nnz, &flags,
                                     ctx->st);
  cudaStreamSynchronize(ctx->st);
  scratch.release();
  if (e != cudaSuccess) {
    p->bufs.release();
    delete p;
    return set_err(ctx, e == cudaErrorMemoryAllocation ? VD_ENOMEM : VD_ECUDA, "vd_poly_integrate: %s",
                   cudaGetErrorString(e));
  }
  if (flags) {
    p->bufs.release();
    delete p;
    return set_err(ctx, VD_EDEGENERATE, "vd_poly_integrate: an edge without two vertices (flags %u)", flags);
  }
  *out = p;
  return VD_OK;
}

vd_status vd_poly_get(const vd_poly* p, double* V, double* F, int64_t* nnz, int64_t* rowptr, int32_t* col,
                      double* A, double* Fd, int32_t on_device) {
  if (!p) return VD_EINVAL;
  if (nnz) *nnz = p->nnz;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (dst && bytes && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, k, p->st);
  };
  cp(V, p->V, (size_t)p->N * sizeof(double));
  cp(F, p->F, (size_t)p->N * sizeof(double));
  cp(rowptr, p->rowptr, (size_t)(p->N + 1) * sizeof(int64_t));
  cp(col, p->col, (size_t)p->nnz * sizeof(int32_t));
  cp(A, p->A, (size_t)p->nnz * sizeof(double));
  cp(Fd, p->Fd, (size_t)p->nnz * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  return e == cudaSuccess ? VD_OK : VD_ECUDA;
}

void vd_poly_free(vd_poly* p) {
  if (!p) return;
  cudaStreamSynchronize(p->st);
  p->bufs.release();
  delete p;
}

void vd_mc_free(vd_mc* mc) {
  if (!mc) return;
  cudaStreamSynchronize(mc->st);
  mc->bufs.release();
  delete mc;
}

namespace vd {
__global__ void k_gather_nnz(const SetDesc* sets, int nsets, int64_t* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsets) out[s] = sets[s].rowptr[sets[s].tv.N];
}
}  // namespace vd

vd_status vd_mc_integrate_batch(vd_ctx* ctx, int32_t nsets, const double* const* X, const int64_t* N,
                                const int32_t* d, int64_t R, uint64_t seed, vd_mc** out, int32_t on_device) {
  if (!ctx || nsets < 0 || (nsets > 0 && (!X || !N || !d || !out))) return VD_EINVAL;
  if (!ctx->cfg.box) return set_err(ctx, VD_EINVAL, "vd_mc_integrate_batch: needs box clipping");
  if (R < 1 || R > ((int64_t)1 << 31)) return set_err(ctx, VD_EINVAL, "vd_mc_integrate_batch: bad rays_per_cell");
  for (int s = 0; s < nsets; ++s) {
    out[s] = nullptr;
    if (!X[s] || N[s] < 1 || N[s] > ((int64_t)1 << 30) || d[s] < 1 || d[s] > 8)
      return set_err(ctx, VD_EINVAL, "vd_mc_integrate_batch: set %d needs 1 <= N <= 2^30 and 1 <= d <= 8", s);
  }
  if (nsets == 0) return VD_OK;
  std::vector<vd_mc*> mcs(nsets, nullptr);
  std::vector<vd::SetDesc> desc(nsets);
  // Device memory in two blocks instead of ~25 allocations per set: the
  // results every set keeps (X, per-ray hits and lengths, V, CSR) in one
  // block shared by the sets' vd_mc objects (freed with the last of them),
  // and everything only the forward pass needs (trees, candidate lists,
  // counts, work lists) in a per-context arena reused by later calls.
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  std::vector<int> Ks(nsets);
  std::vector<size_t> prep_set(nsets);
  size_t keep_bytes = 0;
  for (int s = 0; s < nsets; ++s) {
    const int64_t n = N[s];
    const int dd = d[s];
    Ks[s] = (int)std::min<int64_t>(std::max(vd::default_knn_k(dd), 1), std::max<int64_t>(n - 1, 1));
    const int64_t cap = n * std::min<int64_t>(R, n - 1 + 2 * dd);
    keep_bytes += al(n * dd * 8) + al(n * R * 4) + al(n * R * 8) + al(n * 8) + al((n + 1) * 8) +
                  al(std::max<int64_t>(cap, 1) * 4) + al(std::max<int64_t>(cap, 1) * 8);
    const int64_t ntl = (n + 31) / 32;
    prep_set[s] = al(ntl * 32 * dd * 12) + al(ntl * 32 * 4) + 2 * al((ntl + ntl / 16 + 8) * dd * 24) +
                  al(n * 24 + 65536) + al(n * 8) * 2 + al(n * 4) * 2 + al((size_t)n * Ks[s] * 4) + al(n * 8) +
                  al(n * dd * 4) + al(n * 8) + 40 * 256;
  }
  void* keep_base = nullptr;
  if (cudaMalloc(&keep_base, keep_bytes) != cudaSuccess)
    return set_err(ctx, VD_ENOMEM, "vd_mc_integrate_batch: %zu bytes for the results", keep_bytes);
  std::shared_ptr<void> keep(keep_base, [](void* p) { cudaFree(p); });
  vd::Arena keep_arena{static_cast<char*>(keep_base), keep_bytes, 0};
  // set preparation runs on several host threads, each with its own stream
  // and its own slice of the arena (the tree and list builds wait on the
  // device a few times per set; threads overlap those waits)
  const int T = std::max(1, std::min(nsets, 8));
  std::vector<size_t> slice(T, (size_t)1 << 16);
  for (int s = 0; s < nsets; ++s) slice[s % T] += prep_set[s];
  size_t prep_bytes = 0;
  for (int t = 0; t < T; ++t) prep_bytes += al(slice[t]);
  char* prep_base = nullptr;
  {
    void* pb = nullptr;
    if (ctx->batch_ws.get(0, prep_bytes, &pb) == cudaSuccess) prep_base = static_cast<char*>(pb);
  }
  std::vector<vd::Arena> arenas(T);
  std::vector<DevBufs> preps(T);
  {
    size_t off = 0;
    for (int t = 0; t < T; ++t) {
      if (prep_base) arenas[t] = vd::Arena{prep_base + off, slice[t], 0};
      off += al(slice[t]);
      preps[t].arena = &arenas[t];
    }
  }
  vd::Arena misc_arena;  // descriptors and work lists, after the per-thread slices
  DevBufs prep;          // owns whatever outgrew an arena; freed at the end
  struct PrepGuard {
    DevBufs& b;
    std::vector<DevBufs>& v;
    cudaStream_t st;
    ~PrepGuard() {
      cudaStreamSynchronize(st);
      b.release();
      for (auto& x : v) x.release();
    }
  } prep_guard{prep, preps, ctx->st};
  auto fail = [&](vd_status st) {
    cudaStreamSynchronize(ctx->st);
    for (vd_mc* m : mcs)
      if (m) {
        m->bufs.release();
        delete m;
      }
    return st;
  };
  ctx->last = vd_stats{};
  const long long l0 = vd::g_launches.load();
  int64_t nitems = 0;
  int maxK = 1, maxd = 1;
  // results: carved from the shared block in set order
  for (int s = 0; s < nsets; ++s) {
    vd_mc* mc = new (std::nothrow) vd_mc();
    if (!mc) return fail(VD_ENOMEM);
    mcs[s] = mc;
    const int64_t n = N[s];
    const int dd = d[s];
    mc->st = ctx->st;
    mc->N = n;
    mc->d = dd;
    mc->R = R;
    mc->seed = seed;
    mc->set = (uint32_t)s;
    mc->pool = keep;
    const int64_t cap = n * std::min<int64_t>(R, n - 1 + 2 * dd);
    DevBufs kb;
    kb.arena = &keep_arena;
    cudaError_t e = kb.alloc_n(&mc->X, (size_t)n * dd);
    if (e == cudaSuccess) e = kb.alloc_n(&mc->hit, (size_t)n * R);
    if (e == cudaSuccess) e = kb.alloc_n(&mc->l, (size_t)n * R);
    if (e == cudaSuccess) e = kb.alloc_n(&mc->V, (size_t)n);
    if (e == cudaSuccess) e = kb.alloc_n(&mc->rowptr, (size_t)n + 1);
    if (e == cudaSuccess) e = kb.alloc_n(&mc->col, (size_t)std::max<int64_t>(cap, 1));
    if (e == cudaSuccess) e = kb.alloc_n(&mc->A, (size_t)std::max<int64_t>(cap, 1));
    mc->bufs.ptrs = kb.ptrs;  // empty unless the block was too small
    if (e != cudaSuccess) return fail(cuda_err(ctx, e, "vd_mc_integrate_batch: result buffers"));
    const double S = 2.0 * std::pow(M_PI, 0.5 * dd) / std::tgamma(0.5 * dd);
    vd::SetDesc& D = desc[s];
    D.item0 = nitems;
    D.set = (uint32_t)s;
    D.hit = mc->hit;
    D.l = mc->l;
    D.V = mc->V;
    D.rowptr = mc->rowptr;
    D.col = mc->col;
    D.A = mc->A;
    D.cV = S / ((double)dd * (double)R);
    D.cA = S / (double)R;
    nitems += n;
    maxd = std::max(maxd, dd);
  }
  // node preparation of every set (tree + candidate lists)
  std::vector<cudaError_t> terr(T, cudaSuccess);
  std::vector<int> tbad(T, -1);
  cudaStreamSynchronize(ctx->st);
  auto work = [&](int t) {
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (int s = t; s < nsets && e == cudaSuccess; s += T) {
      vd_mc* mc = mcs[s];
      e = cudaMemcpyAsync(mc->X, X[s], (size_t)mc->N * mc->d * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
      TreeView tv;
      if (e == cudaSuccess) e = vd::build_tree(mc->X, mc->N, mc->d, st, preps[t], &tv);
      if (e == cudaSuccess) e = vd::build_knn(&tv, Ks[s], st, preps[t]);
      int64_t* cnt = nullptr;
      if (e == cudaSuccess) e = preps[t].alloc_n(&cnt, (size_t)mc->N);
      desc[s].tv = tv;
      desc[s].cnt = cnt;
      if (e != cudaSuccess) tbad[t] = s;
    }
    if (st) {
      const cudaError_t e2 = cudaStreamSynchronize(st);
      if (e == cudaSuccess) e = e2;
      cudaStreamDestroy(st);
    }
    terr[t] = e;
  };
  {
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
  }
  for (int t = 0; t < T; ++t) {
    if (terr[t] == cudaErrorInvalidValue)
      return fail(set_err(ctx, VD_EINVAL, "set %d: non-finite coordinate", tbad[t]));
    if (terr[t] != cudaSuccess) return fail(cuda_err(ctx, terr[t], "vd_mc_integrate_batch: set preparation"));
  }
  for (int s = 0; s < nsets; ++s) maxK = std::max(maxK, desc[s].tv.K);
  {  // descriptors and per-set work lists from one more block
    size_t mb = al(nsets * sizeof(vd::SetDesc)) + al(nsets * 8) + al(nsets * sizeof(Counters)) + 4096;
    for (int s = 0; s < nsets; ++s) {
      const int64_t rays = mcs[s]->N * R;
      mb += 2 * al(std::max<int64_t>(rays / 4, 1024) * 4) + al(std::max<int64_t>(rays / 16, 1024) * 4);
    }
    void* p = nullptr;
    if (ctx->batch_ws.get(1, mb, &p) == cudaSuccess) misc_arena = vd::Arena{static_cast<char*>(p), mb, 0};
    prep.arena = &misc_arena;
  }
  DevBufs& tmp = prep;
  vd::SetDesc* desc_dev = nullptr;
  int64_t* nnz_dev = nullptr;
  Counters* set_ctr = nullptr;
  cudaError_t e = tmp.alloc_n(&desc_dev, nsets);
  if (e == cudaSuccess) e = tmp.alloc_n(&nnz_dev, nsets);
  if (e == cudaSuccess) e = tmp.alloc_n(&set_ctr, nsets);
  for (int s = 0; s < nsets && e == cudaSuccess; ++s) {
    vd::SetDesc& D = desc[s];
    const int64_t rays = mcs[s]->N * R;
    D.ctr = set_ctr + s;
    D.fb_cap = std::max<int64_t>(rays / 4, 1024);
    D.ov_cap = std::max<int64_t>(rays / 16, 1024);
    if (e == cudaSuccess) e = tmp.alloc_n(&D.fb_cell, D.fb_cap);
    if (e == cudaSuccess) e = tmp.alloc_n(&D.fb_ray, D.fb_cap);
    if (e == cudaSuccess) e = tmp.alloc_n(&D.ov_list, D.ov_cap);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(desc_dev, desc.data(), nsets * sizeof(vd::SetDesc), cudaMemcpyHostToDevice, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) return fail(cuda_err(ctx, e, "vd_mc_integrate_batch: descriptors"));
  // the forward pass runs as one CUDA graph on a private stream (the context
  // stream may be the legacy default stream, which cannot be captured)
  cudaStream_t gs = nullptr;
  cudaEvent_t ev = nullptr, ga = nullptr, gb = nullptr;
  e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e == cudaSuccess) e = cudaEventCreate(&ga);
  if (e == cudaSuccess) e = cudaEventCreate(&gb);
  struct StreamGuard {
    cudaStream_t s;
    cudaEvent_t a, b, c;
    ~StreamGuard() {
      if (s) cudaStreamDestroy(s);
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      if (c) cudaEventDestroy(c);
    }
  } sg{gs, ev, ga, gb};
  if (e != cudaSuccess) return fail(cuda_err(ctx, e, "vd_mc_integrate_batch: stream"));
  // autotuner: threads per block of the persistent kernel, per largest d,
  // timed on the first cells of the batch (a few per resident block)
  int& threads = ctx->batch_threads[std::min(maxd, 8)];
  if (threads == 0) {
    float best = INFINITY;
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t sample = std::min<int64_t>(nitems, (int64_t)nsm * 64);
    for (int th : {64, 128, 256}) {
      cudaEventRecord(ga, gs);
      e = vd::launch_mc_batch_cells(desc_dev, desc.data(), nsets, sample, maxK, R, seed, th, ctx->ctr, gs);
      cudaEventRecord(gb, gs);
      if (e == cudaSuccess) e = cudaEventSynchronize(gb);
      if (e != cudaSuccess) return fail(cuda_err(ctx, e, "vd_mc_integrate_batch: autotune"));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ga, gb);
      if (ms < best) {
        best = ms;
        threads = th;
      }
    }
  }
  cudaGraph_t graph = nullptr;
  cudaEventRecord(ev, ctx->st);
  cudaStreamWaitEvent(gs, ev, 0);
  e = cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), gs);
    cudaError_t e2 =
        vd::launch_mc_batch(desc_dev, desc.data(), nsets, nitems, maxd, maxK, R, seed, threads, ctx->ctr, gs);
    e = cudaStreamEndCapture(gs, &graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && ctx->batch_exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ctx->batch_exec, graph, &info) != cudaSuccess) {
      cudaGetLastError();  // another shape: instantiate below
      cudaGraphExecDestroy(ctx->batch_exec);
      ctx->batch_exec = nullptr;
    }
  }
  if (e == cudaSuccess && !ctx->batch_exec) e = cudaGraphInstantiate(&ctx->batch_exec, graph, 0);
  if (e == cudaSuccess) {
    cudaEventRecord(ga, gs);
    e = cudaGraphLaunch(ctx->batch_exec, gs);
    cudaEventRecord(gb, gs);
  }
  if (e == cudaSuccess) {
    vd::k_gather_nnz<<<(nsets + 127) / 128, 128, 0, gs>>>(desc_dev, nsets, nnz_dev);
    vd::count_launch();
    e = cudaGetLastError();
  }
  std::vector<int64_t> nnz(nsets);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nnz.data(), nnz_dev, nsets * sizeof(int64_t), cudaMemcpyDeviceToHost, gs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(gs);
  float gms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&gms, ga, gb);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(cuda_err(ctx, e, "vd_mc_integrate_batch: graph"));
  Counters hc;
  vd_status st2 = read_counters(ctx, &hc);
  if (st2 == VD_OK) st2 = check_flags(ctx, hc);
  if (st2 != VD_OK) return fail(st2);
  std::vector<Counters> hs(nsets);
  e = cudaMemcpy(hs.data(), set_ctr, nsets * sizeof(Counters), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(cuda_err(ctx, e, "vd_mc_integrate_batch: counters"));
  int64_t nfb = 0;
  for (int s = 0; s < nsets; ++s) {
    if ((st2 = check_flags(ctx, hs[s])) != VD_OK) return fail(st2);
    if ((int64_t)hs[s].fallback > desc[s].fb_cap || (int64_t)hs[s].overflow > desc[s].ov_cap)
      return fail(set_err(ctx, VD_EOVERFLOW, "set %d: work list overflow", s));
    nfb += (int64_t)hs[s].fallback;
    hc.pairs += hs[s].pairs;
  }
  hc.aux0 = (unsigned long long)nfb;
  for (int s = 0; s < nsets; ++s) {
    mcs[s]->nnz = nnz[s];
    mcs[s]->stats.rays = mcs[s]->N * R;
    out[s] = mcs[s];
  }
  ctx->last.rays = nitems * R;
  ctx->last.pairs_screened = (int64_t)hc.pairs;
  ctx->last.rechecked = (int64_t)hc.rechecked;
  ctx->last.fallback_rays = (int64_t)hc.aux0;
  ctx->last.ms = gms;
  ctx->last.raycast_ms = gms;
  ctx->last.launches = vd::g_launches.load() - l0;
  return VD_OK;
}

// ------------------------------------------------------------- vertices --
vd_status vd_random_walk(vd_ctx* ctx, const int32_t* start, int64_t W, int64_t steps, uint64_t seed,
                         int32_t* path_tuples, double* path_coords, int32_t on_device) {
  if (!ctx || (W > 0 && (!start || !path_tuples)) || W < 0 || steps < 0) return VD_EINVAL;
  if (!ctx->X) return set_err(ctx, VD_EINVAL, "vd_random_walk: no node set");
  if (!ctx->cfg.box) return set_err(ctx, VD_EINVAL, "vd_random_walk: needs box clipping");
  if (ctx->d < 2 || ctx->d > 6) return set_err(ctx, VD_EINVAL, "vd_random_walk: needs 2 <= d <= 6");
  if (W > ((int64_t)1 << 30) || steps > ((int64_t)1 << 31))
    return set_err(ctx, VD_EINVAL, "vd_random_walk: too many walkers or steps");
  const int d = ctx->d, L = d + 1;
  DevBufs tmp;
  const int32_t* st_d = start;
  int32_t* pt = path_tuples;
  double* px = path_coords;
  cudaError_t e = cudaSuccess;
  if (!on_device && W > 0) {
    int32_t* s2 = nullptr;
    e = tmp.alloc_n(&s2, (size_t)W * L);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s2, start, (size_t)W * L * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->st);
    st_d = s2;
    if (e == cudaSuccess) e = tmp.alloc_n(&pt, (size_t)std::max<int64_t>(W * steps, 1) * L);
    if (e == cudaSuccess && path_coords) e = tmp.alloc_n(&px, (size_t)std::max<int64_t>(W * steps, 1) * d);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), ctx->st);
  double rms = 0.0;
  Timer tm(ctx->st);
  if (e == cudaSuccess)
    e = vd::random_walk(ctx->tree, effective_precision(ctx), st_d, W, steps, seed, pt, px, ctx->ctr, tmp, ctx->st, &rms);
  const double ms = tm.stop();
  if (e == cudaSuccess && !on_device && W > 0) {
    e = cudaMemcpyAsync(path_tuples, pt, (size_t)W * steps * L * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess && path_coords)
      e = cudaMemcpyAsync(path_coords, px, (size_t)W * steps * d * sizeof(double), cudaMemcpyDeviceToHost, ctx->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  cudaStreamSynchronize(ctx->st);
  tmp.release();
  if (e != cudaSuccess) return cuda_err(ctx, e, "vd_random_walk");
  Counters hc;
  vd_status s = read_counters(ctx, &hc);
  if (s == VD_OK) s = check_flags(ctx, hc);
  if (s == VD_OK) {
    vd_stats st{};
    st.rays = W * steps;
    st.ms = ms;
    st.raycast_ms = rms;
    st.rechecked = (int64_t)hc.rechecked;
    st.pairs_screened = (int64_t)hc.pairs;
    ctx->last = st;
  }
  return s;
}

// The whole-diagram traversal (cells_per_batch = 0) or the per-cell
// exploration in batches of cells_per_batch cells.
static vd_status vertices_impl(vd_ctx* ctx, int64_t cells_per_batch, vd_mesh** out) {
  if (!ctx || !out) return VD_EINVAL;
  *out = nullptr;
  if (!ctx->X) return set_err(ctx, VD_EINVAL, "vd_vertices: no node set");
  if (!ctx->cfg.box) return set_err(ctx, VD_EINVAL, "vd_vertices: needs box clipping");
  if (ctx->N < 1) return set_err(ctx, VD_EINVAL, "vd_vertices: empty node set");
  vd_mesh* m = new (std::nothrow) vd_mesh();
  if (!m) return VD_ENOMEM;
  m->bufs.cache = ctx->result_cache;
  m->st = ctx->st;
  m->d = ctx->d;
  VD_CK(cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), ctx->st), "memset");
  const long long l0 = vd::g_launches.load();
  Timer tm(ctx->st);
  char err[256] = {0};
  cudaError_t e = vd::traverse_vertices(ctx->tree, effective_precision(ctx), ctx->cfg, cells_per_batch, ctx->trav_ws,
                                        m->bufs, &m->tuples, &m->coords, &m->nv, &m->stats, ctx->ctr, ctx->st, err,
                                        sizeof(err));
  m->stats.ms = tm.stop();
  m->stats.launches = vd::g_launches.load() - l0;
  Counters hc;
  vd_status s = VD_OK;
  if (e != cudaSuccess) {
    s = err[0] ? set_err(ctx, VD_EDEGENERATE, "vd_vertices: %s", err) : cuda_err(ctx, e, "vd_vertices");
  } else {
    s = read_counters(ctx, &hc);
    if (s == VD_OK) s = check_flags(ctx, hc);
    if (s == VD_OK) {
      m->stats.rechecked = (int64_t)hc.rechecked;
      m->stats.tiles_visited = (int64_t)hc.tiles;
      m->stats.pairs_screened = (int64_t)hc.pairs;
    }
  }
  if (s != VD_OK) {
    cudaStreamSynchronize(ctx->st);
    m->bufs.release();
    delete m;
    return s;
  }
  ctx->last = m->stats;
  *out = m;
  return VD_OK;
}

vd_status vd_vertices(vd_ctx* ctx, vd_mesh** out) { return vertices_impl(ctx, 0, out); }

vd_status vd_vertices_by_cells(vd_ctx* ctx, int64_t cells_per_batch, vd_mesh** out) {
  if (!ctx || !out) return VD_EINVAL;
  if (cells_per_batch < 0) return set_err(ctx, VD_EINVAL, "vd_vertices_by_cells: negative batch size");
  const int64_t b = cells_per_batch > 0 ? cells_per_batch : std::max<int64_t>(1, (ctx->N + 15) / 16);
  return vertices_impl(ctx, b, out);
}

int64_t vd_mesh_count(const vd_mesh* m) { return m ? m->nv : 0; }
int32_t vd_mesh_dim(const vd_mesh* m) { return m ? m->d : 0; }

vd_status vd_mesh_copy(const vd_mesh* m, int32_t* tuples, double* coords, int32_t on_device) {
  if (!m) return VD_EINVAL;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  if (tuples && m->nv) e = cudaMemcpyAsync(tuples, m->tuples, m->nv * (m->d + 1) * sizeof(int32_t), k, m->st);
  if (coords && m->nv && e == cudaSuccess)
    e = cudaMemcpyAsync(coords, m->coords, m->nv * m->d * sizeof(double), k, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  return e == cudaSuccess ? VD_OK : VD_ECUDA;
}

vd_status vd_mesh_stats(const vd_mesh* m, vd_stats* out) {
  if (!m || !out) return VD_EINVAL;
  *out = m->stats;
  return VD_OK;
}

void vd_mesh_free(vd_mesh* m) {
  if (!m) return;
  cudaStreamSynchronize(m->st);
  m->bufs.release();
  delete m;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free RayCast.  Some callers cannot let a library call cudaMalloc
// on their hot path: their device memory belongs to another allocator (a
// framework's caching pool or an arena sized once at start-up), or they run a
// steady-state loop that must not pay cudaMalloc's implicit synchronisation or
// risk an out-of-memory error mid-run.  vd_raycast_noalloc serves them: its
// work lists and counters live in the file-scope device array below, so the
// call itself allocates nothing.  The array is the same for every call and
// every context in the process and holds the previous call's contents: the
// counters are cleared at the start of each call, and two calls that overlap
// on the GPU (other streams or threads) race on it.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxRays = (int64_t)1 << 18;  // 262,144 rays per call

struct NoAllocScratch {
  Counters ctr;
  int32_t overflow[kNoAllocMaxRays];  // rays redone on the binary64 path
  int32_t fallback[kNoAllocMaxRays];  // rays finished by the tree walk
};

// 2 MiB (+ counters), resident on every device that loads the library.
__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of the scratch array for this call.  Host code only sees a
// host-side stand-in under the array's name, so the address is looked up on
// every call, with the context's device current: a cached address would go
// stale once the device's context is torn down and created again (for
// example after cudaDeviceReset), and a kernel given it would fault.
vd_status noalloc_scratch(vd_ctx* ctx, NoAllocScratch** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(ctx, e, "vd_raycast_noalloc: cudaGetDevice");
  if (dev != ctx->dev)
    return set_err(ctx, VD_EINVAL, "vd_raycast_noalloc: the current device %d is not the context's device %d", dev,
                   ctx->dev);
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) return cuda_err(ctx, e, "vd_raycast_noalloc: cudaGetSymbolAddress");
  *out = static_cast<NoAllocScratch*>(p);
  return VD_OK;
}

}  // namespace

extern "C" vd_status vd_raycast_noalloc(vd_ctx* ctx, const double* origins, const double* dirs, const int32_t* eta,
                                        int32_t eta_stride, int64_t R, int32_t* hit, double* t) {
  if (!ctx) return VD_EINVAL;
  if (!ctx->X) return set_err(ctx, VD_EINVAL, "vd_raycast_noalloc: no node set");
  if (R < 0 || (R > 0 && (!origins || !dirs || !eta || !hit || !t)) || eta_stride < 1 || eta_stride > ctx->d + 1)
    return set_err(ctx, VD_EINVAL, "vd_raycast_noalloc: bad arguments (R=%lld, eta_stride=%d, d=%d)",
                   (long long)R, eta_stride, ctx->d);
  if (R > kNoAllocMaxRays)
    return set_err(ctx, VD_EINVAL, "vd_raycast_noalloc: R=%lld exceeds the fixed scratch limit of %lld rays",
                   (long long)R, (long long)kNoAllocMaxRays);
  ctx->last = vd_stats{};
  if (R == 0) return VD_OK;
  NoAllocScratch* sc = nullptr;
  vd_status s = noalloc_scratch(ctx, &sc);
  if (s != VD_OK) return s;
  vd::RaySource rs;
  rs.mode = 0;
  rs.R = R;
  rs.origins = origins;
  rs.dirs = dirs;
  rs.eta = eta;
  rs.eta_stride = eta_stride;
  rs.box = ctx->cfg.box;
  vd::RayOut ro;
  ro.hit = hit;
  ro.t = t;
  ro.overflow_list = sc->overflow;
  ro.overflow_cap = kNoAllocMaxRays;
  ro.fallback_list = sc->fallback;
  ro.fallback_cap = kNoAllocMaxRays;
  VD_CK(cudaMemsetAsync(&sc->ctr, 0, sizeof(Counters), ctx->st), "vd_raycast_noalloc: clear counters");
  int64_t nfb = 0;
  VD_CK(vd::launch_raycast(ctx->tree, rs, ro, effective_precision(ctx), &sc->ctr, ctx->st, &nfb),
        "vd_raycast_noalloc");
  Counters hc;
  VD_CK(cudaMemcpyAsync(&hc, &sc->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->st), "counters");
  VD_CK(cudaStreamSynchronize(ctx->st), "sync");
  ctx->last.rays = R;
  ctx->last.tiles_visited = (int64_t)hc.tiles;
  ctx->last.pairs_screened = (int64_t)hc.pairs;
  ctx->last.rechecked = (int64_t)hc.rechecked;
  ctx->last.overflow_rays = (int64_t)hc.overflow;
  ctx->last.fallback_rays = nfb;
  return check_flags(ctx, hc);
}
