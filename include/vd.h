/*
 * vd.h -- C ABI of libvd: the exact Voronoi RayCast, the exhaustive vertex
 * traversal and the Monte Carlo cell integrals with their adjoint, after
 * Sikorski & Heida, "Voronoi Graph: improved raycasting and integration
 * schemes for high dimensional Voronoi diagrams" (arXiv 2405.10050).
 * Everything runs on one CUDA GPU (sm_103a).
 *
 * Conventions used by every entry point
 *  - Nodes X: N x d float64, row-major, 1 <= d <= 16, N >= 1.
 *  - Generator ids: nodes 0..N-1; the 2d faces of the unit box [0,1]^d are
 *    pseudo-generators with negative ids -(2a+s+1) for axis a, side s
 *    (s = 0: x_a = 0, s = 1: x_a = 1).  VD_NO_ID (INT32_MIN) means "none".
 *  - Pointers: the trailing `on_device` argument says whether the array
 *    arguments of that call are device pointers (1) or host pointers (0).
 *    Host pointers are copied on the context's stream and the call returns
 *    after the copies finish.  Device pointers must stay valid until the
 *    call returns (every call synchronises its stream before returning).
 *  - Ownership: the caller owns every array it passes; library objects
 *    (vd_ctx, vd_mesh, vd_mc) are owned by the library until their free call.
 *  - Device memory: freeing a vd_mesh or (unbatched) vd_mc hands its device
 *    blocks to its context, which reuses them for its next results (up to
 *    16 GiB are kept); they are returned to CUDA when the context and the
 *    last of its results are freed.  A context keeps one block for its node
 *    set, sized by the largest node set so far.
 *  - Errors: every call returns a vd_status and throws nothing across the
 *    ABI; vd_last_error() gives a message for the last failure on a context.
 *  - Floating point: the exact path (VD_FP64) and the recheck of the mixed
 *    paths evaluate t in binary64 in one canonical operation order, so hit
 *    ids are identical across precisions and against an FP64 reference that
 *    follows the same order.
 */
#ifndef VD_H
#define VD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VD_NO_ID INT32_MIN
#define VD_MAX_D 16

typedef enum {
  VD_OK = 0,
  VD_EINVAL = -1,      /* bad argument (size, dimension, pointer, state)   */
  VD_ENOMEM = -2,      /* device or host allocation failed                 */
  VD_ECUDA = -3,       /* a CUDA runtime call failed                       */
  VD_EDEGENERATE = -4, /* duplicate nodes or a degenerate solve            */
  VD_EHASHFULL = -5,   /* traversal hash or vertex table capacity reached  */
  VD_EOVERFLOW = -6,   /* a bounded work list overflowed                   */
  VD_ETIMEOUT = -7     /* a bounded device-side wait gave up               */
} vd_status;

typedef enum {
  VD_FP64 = 0,  /* every (ray, node) pair in binary64                      */
  VD_FP32 = 1,  /* binary32 screening with a proven error margin, binary64
                   recheck of the survivors                                */
  VD_TC16 = 2,  /* dot products on the tensor cores (tcgen05, fp16 in,
                   fp32 accumulate) with a proven error margin, binary64
                   recheck: MC rays (cell lists, or the block tree walk
                   without lists) and explicit rays with candidate lists
                   (vd_raycast, vd_vertices, vd_random_walk; rays grouped
                   by reference node); other calls treat it as VD_FP32   */
  VD_AUTO = 3   /* per call, the path measured fastest on GB300: VD_TC16
                   for MC rays of node sets without candidate lists
                   (d > 8) and for explicit rays with candidate lists at
                   3 <= d <= 8, VD_FP32 otherwise; results are identical
                   on every path                                        */
} vd_precision;

typedef struct {
  int32_t precision;      /* vd_precision, default VD_AUTO                  */
  int32_t box;            /* 1: clip cells to [0,1]^d (required by vertices
                             and MC); 0: unbounded rays may miss           */
  int64_t hash_capacity;  /* traversal vertex table entries, 0 = automatic */
  int64_t max_levels;     /* traversal BFS level cap, 0 = automatic        */
  int64_t wait_limit;     /* polls before a bounded device wait gives up
                             (VD_ETIMEOUT); 0 = default, < 0 = give up
                             before the first poll (tests that path)       */
  int32_t knn_k;          /* candidate list length per node: 0 = automatic
                             by dimension, -1 = no lists (tree walk only)  */
  int32_t rays_per_block; /* MC rays per thread block, 0 = autotune        */
} vd_config;

typedef struct {
  int64_t rays;            /* rays cast by the last call                    */
  int64_t tiles_visited;   /* node tiles evaluated (all rays)               */
  int64_t pairs_screened;  /* (ray, node) pairs evaluated                   */
  int64_t rechecked;       /* candidates recomputed in binary64             */
  int64_t fallback_rays;   /* MC rays finished by the generic tree search   */
  int64_t overflow_rays;   /* rays recomputed on the plain FP64 path        */
  int64_t ties;            /* exact binary64 ties seen (degenerate input)   */
  int64_t levels;          /* traversal BFS levels                          */
  int64_t vertices;        /* traversal vertices                            */
  int64_t launches;        /* kernels launched by the call                  */
  double ms;               /* device time of the last call, milliseconds   */
  double raycast_ms;       /* device time of its RayCast kernels, ms        */
  int64_t edge_table_bytes;   /* traversal: edge-counter table size, bytes */
  int64_t vertex_table_bytes; /* traversal: vertex table size, bytes       */
} vd_stats;

typedef struct vd_ctx vd_ctx;
typedef struct vd_mesh vd_mesh;
typedef struct vd_mc vd_mc;

/* Number of CUDA kernels libvd has launched in this process (all contexts);
 * a diagnostic counter, never reset. */
int64_t vd_kernel_launches(void);

/* Fills *cfg with the defaults (VD_AUTO, box on, automatic capacities). */
void vd_config_default(vd_config* cfg);

/* Creates a context on the current CUDA device.  cuda_stream is a
 * cudaStream_t (NULL = the legacy default stream); every kernel and copy of
 * the context runs on it.  cfg may be NULL (defaults). */
vd_status vd_create(vd_ctx** ctx, const vd_config* cfg, void* cuda_stream);
void vd_destroy(vd_ctx* ctx);
const char* vd_last_error(const vd_ctx* ctx);
const char* vd_status_str(vd_status s);
vd_status vd_set_precision(vd_ctx* ctx, int32_t precision);
vd_status vd_last_stats(const vd_ctx* ctx, vd_stats* out);

/* Node set (Section 2.1: nodes X in general position).  Copies X and builds
 * the Morton-ordered node tiles with their bounding-box hierarchy; the
 * previous node set of the context is released.  EINVAL for N < 1,
 * d outside 1..16, or a non-finite coordinate. */
vd_status vd_set_nodes(vd_ctx* ctx, const double* X, int64_t N, int32_t d, int32_t on_device);

/* RayCast (Section 2.2, Eq. (t), Algorithm 1), R rays.  Ray r starts at
 * origins[r*d..] with unit direction dirs[r*d..]; eta[r*eta_stride..] lists
 * the generators the ray starts equidistant to (they are never returned),
 * padded with VD_NO_ID; eta[r*eta_stride] must be a node, the reference
 * generator g.  Result: the first generator j whose bisector with g the ray
 * crosses, t_j = (|x_j - v|^2 - |g - v|^2) / (2 u.(x_j - g)) minimal over
 * u.(x_j - g) > 0, or the first box face (box on); ties by (t, node before
 * face, id).  hit[r] = VD_NO_ID and t[r] = +inf if nothing is hit.
 * screen_err (nullable): per ray |t_screen - t| / t, the binary32 screening
 * estimate against the binary64 result (0 on the VD_FP64 path). */
vd_status vd_raycast(vd_ctx* ctx, const double* origins, const double* dirs, const int32_t* eta,
                     int32_t eta_stride, int64_t R, int32_t* hit, double* t, float* screen_err,
                     int32_t on_device);

/* Allocation-free variant of vd_raycast (the paper has no counterpart: this
 * is a deployment aid).  For callers that must not have the library call
 * cudaMalloc while they run -- their device memory belongs to another
 * allocator, or a steady-state loop must not pay cudaMalloc's implicit
 * synchronisation or risk running out of memory mid-run.  Same arguments and
 * results as vd_raycast, except: origins, dirs, eta, hit and t must be DEVICE
 * pointers; screen_err is not produced; R <= 262,144 (larger R returns
 * VD_EINVAL).  Its work lists and counters live in one fixed 2 MiB device
 * array inside libvd (resident on every GPU that loads the library until the
 * process exits), shared by all calls and contexts: calls that overlap on the
 * GPU race on it.  Each call looks up that array's address on the current
 * device, which must be the context's device (VD_EINVAL otherwise), and waits
 * for the context's stream before it returns.  The context must already hold
 * a node set (vd_set_nodes, which does allocate); this call itself allocates
 * nothing. */
vd_status vd_raycast_noalloc(vd_ctx* ctx, const double* origins, const double* dirs, const int32_t* eta,
                             int32_t eta_stride, int64_t R, int32_t* hit, double* t);

/* Exhaustive vertex traversal (Section 2.3, Algorithm 2) of the diagram
 * clipped to [0,1]^d: seeds by Descent, then casts one ray along every edge
 * whose second vertex is still unknown, deduplicating vertices by their sorted
 * (d+1)-generator tuple.  Box must be on.  EHASHFULL if the vertex table
 * capacity is reached. */
vd_status vd_vertices(vd_ctx* ctx, vd_mesh** out);

/* Per-cell sequential exploration (Section 2.3: the cells are explored in
 * sequential order so that the edge counts are reconstructed for each cell
 * and the edge table holds only the current cells' edges).  Cells are taken
 * in index order, cells_per_batch at a time (1 = one cell at a time; 0 =
 * automatic, N / 16).  For each batch the edge counters are rebuilt from the
 * vertices found so far (edges that hold a batch node only), batch cells
 * without a known vertex are seeded by Descent, and the traversal follows
 * only edges that hold a batch node.  Same result as vd_vertices (the same
 * vertex set, tuples and coordinates bit for bit); stats report both tables'
 * sizes.  EDEGENERATE if a cell ends a batch without a vertex. */
vd_status vd_vertices_by_cells(vd_ctx* ctx, int64_t cells_per_batch, vd_mesh** out);
int64_t vd_mesh_count(const vd_mesh* mesh);
int32_t vd_mesh_dim(const vd_mesh* mesh);
/* tuples: V x (d+1) int32, each row ascending, rows in lexicographic order;
 * coords: V x d float64 (solved from the tuple).  Either may be NULL. */
vd_status vd_mesh_copy(const vd_mesh* mesh, int32_t* tuples, double* coords, int32_t on_device);
vd_status vd_mesh_stats(const vd_mesh* mesh, vd_stats* out);
void vd_mesh_free(vd_mesh* mesh);

/* Random walks on the vertex graph (Section 2.3: the random walk that
 * approximates the Voronoi graph, here with the incircle RayCast), 2 <= d
 * <= 6, box on.  Walker w starts at the vertex with sorted tuple
 * start[w] (W x (d+1) int32, a vertex of the context's diagram); at each
 * step it takes one of its vertex's edges that hold a node, drawn by
 * Philox4x32-10 at counter (step, w, 0x57414C4B, 0), key (seed): with the
 * valid drop indices a_0 < ... < a_{n-1} of the tuple it takes a_k,
 * k = (word0 n) >> 32; it casts the ray along that edge (SearchDirection,
 * reference node first) and moves to the far vertex.  path_tuples: W x steps
 * x (d+1) sorted tuples; path_coords: W x steps x d float64 (may be NULL).
 * VD_EDEGENERATE if a step met a degenerate solve (that walker stays put).
 * vd_last_stats: rays = W * steps, ms, raycast_ms. */
vd_status vd_random_walk(vd_ctx* ctx, const int32_t* start, int64_t W, int64_t steps, uint64_t seed,
                         int32_t* path_tuples, double* path_coords, int32_t on_device);

/* Monte Carlo volumes and interface areas (Section 3.1, Algorithm 3) of all
 * N cells with R rays per cell.  Ray k of cell i has the direction drawn by
 * vd_mc_directions (Philox4x32-10 keyed by seed) and is cast from x_i with
 * eta = {i}; l_k = t*.  V_i = S_{d-1}/(dR) sum_k l_k^d and
 * A_ij = S_{d-1}/R sum_{k: hit j} l_k^{d-1} / |n_ij . u_k|.  The per-ray
 * (hit, l) are kept for the adjoint.  Box must be on. */
vd_status vd_mc_integrate(vd_ctx* ctx, int64_t rays_per_cell, uint64_t seed, vd_mc** out);
/* V: N float64.  Row i of the CSR (rowptr N+1 int64, col/A nnz) lists the
 * distinct generators hit from cell i in ascending id order (faces first).
 * *nnz is always written; rowptr/col/A may be NULL to query nnz. */
vd_status vd_mc_get(const vd_mc* mc, double* V, int64_t* nnz, int64_t* rowptr, int32_t* col, double* A,
                    int32_t on_device);
/* Saved per-ray results: hit N*R int32 and l N*R float64, ray (i,k) at i*R+k. */
vd_status vd_mc_rays(const vd_mc* mc, int32_t* hit, double* l, int32_t on_device);
/* Adjoint of the estimator with directions and argmins held fixed:
 * gX = sum_i gV_i dV_i/dX + sum_ij gA_ij dA_ij/dX (N x d float64). */
vd_status vd_mc_adjoint(const vd_mc* mc, const double* gV, const double* gA, double* gX, int32_t on_device);
/* Monte Carlo integrals of a function f over the cells (Section 3.1, Eqs.
 * mc-help1 and full_MC_integration, Algorithm 3), from the rays of a
 * finished vd_mc_integrate (its directions, hit ids and lengths):
 *   Fd_ij = S_{d-1}/R sum_{k: hit j} f(r_k) l_k^{d-1} / |n_ij . u_k|,
 *           r_k = x_i + l_k u_k the ray's hit point (f = 1 gives A_ij);
 *   FV_i  = S_{d-1}/(R m) sum_k sum_{s<m} f(x_i + t_ks l_k u_k) t_ks^{d-1} l_k^d,
 *           m samples t_ks ~ U(0,1) along each ray (f = 1 estimates V_i).
 * t_ks = (w + 1/2) 2^-32, w = word (s mod 4) of Philox4x32-10 at counter
 * (2^31 + s div 4, k, i, set), key (seed low, seed high) of the run.
 * Everything in binary64; the sums are deterministic (fixed order).
 * FV: N float64; Fd: nnz float64 in the order of vd_mc_get's col.  Either
 * may be NULL.  m >= 1 (ignored when FV is NULL). */
typedef enum {
  VD_F_ONE = 0,    /* f = 1                                               */
  VD_F_POLY2 = 1,  /* f = c0 + sum_a b[a] y_a + sum_a q[a] y_a^2, binary64,
                      linear terms first, each sum left to right          */
  VD_F_SIN_SQ = 2  /* f = sin(y_axis^2), the integrand of Section 4       */
} vd_func_kind;

typedef struct {
  int32_t kind;           /* vd_func_kind                                   */
  int32_t axis;           /* VD_F_SIN_SQ: 0 <= axis < d                     */
  double c0;              /* VD_F_POLY2 coefficients (entries >= d unused)  */
  double b[VD_MAX_D];
  double q[VD_MAX_D];
} vd_func;

vd_status vd_mc_integrals(const vd_mc* mc, const vd_func* f, int64_t m, double* FV, double* Fd, int32_t on_device);

/* Heuristic Monte Carlo integration (Section 3.3) of the node set of `mc`,
 * from its interface areas A_ij and the vertices of `mesh` (vd_vertices of
 * the same node set):
 *   VH_i = (1/d) sum_j h_ij A_ij  (h_ij = |x_j - x_i|/2, or the distance from
 *          x_i to the box face j);
 *   FH_ij = (d/(d+1)) (1/K_ij) sum_k f(nu_k) A_ij + (1/(d+1)) f(y_ij) A_ij,
 *          nu_k the K_ij vertices whose tuple holds both i and j, y_ij their
 *          mean (0 if the interface has no vertex);
 *   IH_i = sum_j (h_ij/d) ((d/(d+1)) FH_ij + (1/(d+1)) A_ij f(x_i)), the cone
 *          rule of Eq. (leibniz-int) with apex x_i.
 * Binary64, fixed summation orders (k by ascending vertex index, j in CSR
 * order).  VH, IH: N float64; FH: nnz float64 in vd_mc_get's col order; any
 * may be NULL but not all three.  mesh must have the dimension of mc. */
vd_status vd_hmc_integrals(const vd_mc* mc, const vd_mesh* mesh, const vd_func* f, double* VH, double* FH,
                           double* IH, int32_t on_device);
/* Exact cell volumes, interface areas and integrals of the piecewise linear
 * interpolant of f (Section 3.2, Algorithms 4-5) of the context's node set
 * from the vertices of `mesh` (vd_vertices of the same node set), 2 <= d <= 8.
 * Each cell is split into simplices (x_i, m_2, ..., m_{d-1}, nu, nu'): m_D
 * the vertex mean of a level-D face of the cell (level 2 = a facet), nu, nu'
 * an edge of the last face; V_i sums their volumes |det| / d!; the integral
 * is the one of the function that is linear on each simplex and equals f at
 * its corners (Algorithm 5's weights); A_ij = (d / h_ij) times the volume of
 * the pyramid over facet ij, Fd_ij the same for the integral.  Binary64,
 * fixed order (faces by ascending generator, vertices ascending).  Returns
 * VD_EDEGENERATE if an edge of the walk does not have two vertices. */
typedef struct vd_poly vd_poly;
vd_status vd_poly_integrate(vd_ctx* ctx, const vd_mesh* mesh, const vd_func* f, vd_poly** out);
/* V, F: N float64; row i of the CSR (rowptr N+1 int64, col/A/Fd nnz) lists
 * the facets of cell i by ascending generator id (faces first).  *nnz is
 * always written; the arrays may be NULL. */
vd_status vd_poly_get(const vd_poly* p, double* V, double* F, int64_t* nnz, int64_t* rowptr, int32_t* col,
                      double* A, double* Fd, int32_t on_device);
void vd_poly_free(vd_poly* p);
vd_status vd_mc_stats(const vd_mc* mc, vd_stats* out);
int64_t vd_mc_count(const vd_mc* mc);
void vd_mc_free(vd_mc* mc);

/* The directions of rays 0..R-1 of cells cell0..cell0+ncells-1 of point set
 * `set` in dimension d (Section 3.1: a normalised Gaussian draw): out is
 * ncells x R x d float64.  The draw is Philox4x32-10 (Salmon et al. 2011),
 * counter (block, ray, cell, set), key (seed low, seed high); binary32
 * Box-Muller from series-defined log/sin/cos, binary64 normalisation. */
vd_status vd_mc_directions(vd_ctx* ctx, uint64_t seed, uint32_t set, int64_t cell0, int64_t ncells,
                           int64_t R, int32_t d, double* out, int32_t on_device);

/* Batched MC: nsets independent node sets (X[s]: N[s] x d[s], host or
 * device per on_device) in one persistent launch; out[s] receives one
 * vd_mc per set, set s drawing its rays with set id s. */
vd_status vd_mc_integrate_batch(vd_ctx* ctx, int32_t nsets, const double* const* X, const int64_t* N,
                                const int32_t* d, int64_t rays_per_cell, uint64_t seed, vd_mc** out,
                                int32_t on_device);

#ifdef __cplusplus
}
#endif
#endif /* VD_H */
