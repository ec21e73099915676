"""FP64 brute-force CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never loads it.  The arithmetic lives in ``vd_oracle.c``; this
module builds it with gcc and wraps it with ctypes and numpy.  It shares no
code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
NO_ID = -(2**31)

_lib = None


def build(force: bool = False) -> str:
    """Compile vd_oracle.c into liboracle.so (gcc, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, u32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
        L.or_max_threads.restype = ctypes.c_int
        L.or_set_threads.argtypes = [i32]
        L.or_sphere_area.restype = ctypes.c_double
        L.or_sphere_area.argtypes = [i32]
        L.or_log32.restype = ctypes.c_float
        L.or_log32.argtypes = [ctypes.c_float]
        L.or_log32_batch.argtypes = [P, P, i64]
        L.or_sincos2pi24_batch.argtypes = [P, P, P, i64]
        L.or_philox_batch.argtypes = [P, P, P, i64]
        L.or_mc_directions.argtypes = [u64, u32, i64, i64, i64, i32, P]
        L.or_mc_gaussians32.argtypes = [u64, u32, i64, i64, i32, P]
        L.or_raycast.argtypes = [P, i64, i32, i32, P, P, P, i32, i64, P, P]
        L.or_mc_rays.argtypes = [P, i64, i32, i64, u64, u32, P, P]
        L.or_mc_reduce.restype = i64
        L.or_mc_reduce.argtypes = [P, i64, i32, i64, u64, u32, P, P, P, P, P, P, i64]
        L.or_mc_eval_fixed.argtypes = [P, i64, i32, i64, u64, u32, P, P, P, P, P]
        L.or_mc_adjoint.argtypes = [P, i64, i32, i64, u64, u32, P, P, P, P, P, P, P]
        L.or_func_eval.restype = ctypes.c_double
        L.or_func_eval.argtypes = [i32, i32, P, i32, P]
        L.or_mc_tsample.restype = ctypes.c_double
        L.or_mc_tsample.argtypes = [u64, u32, u32, u32, u32]
        L.or_mc_tsamples.argtypes = [u64, u32, i64, i64, i64, P]
        L.or_mc_integrals.argtypes = [P, i64, i32, i64, u64, u32, i64, P, P, P, P, P, i32, i32, P, i64, P, P]
        L.or_hmc.argtypes = [P, i64, i32, P, P, P, P, P, i64, i32, i32, P, P, P, P, P]
        L.or_leibniz.restype = i64
        L.or_leibniz.argtypes = [P, i64, i32, P, P, i64, i32, i32, P, P, P, P, P, P, P, i64]
        L.or_random_walk.restype = ctypes.c_int
        L.or_random_walk.argtypes = [P, i64, i32, P, i64, i64, u64, P, P, P]
        L.or_vertex_coords.restype = ctypes.c_int
        L.or_vertex_coords.argtypes = [P, i32, P, P]
        L.or_search_direction.restype = ctypes.c_int
        L.or_search_direction.argtypes = [P, i32, P, i32, P]
        L.or_descent.restype = ctypes.c_int
        L.or_descent.argtypes = [P, i64, i32, ctypes.c_int32, P]
        L.or_vertices.restype = i64
        L.or_vertices.argtypes = [P, i64, i32, ctypes.c_int32, i64, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(lib().or_max_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on."""
    lib().or_set_threads(int(n))


def sphere_area(d: int) -> float:
    """S_{d-1} = 2 pi^{d/2} / Gamma(d/2) (Section 3.1)."""
    return float(lib().or_sphere_area(d))


def face_id(axis: int, side: int) -> int:
    return -(2 * axis + side + 1)


# --- random numbers --------------------------------------------------------
def philox(ctr: np.ndarray, key) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    lib().or_philox_batch(_p(ctr), _p(k), _p(out), ctr.shape[0])
    return out


def log32(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().or_log32_batch(_p(x), _p(y), x.size)
    return y


def sincos2pi24(a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    c = np.empty(a.shape, np.float32)
    s = np.empty(a.shape, np.float32)
    lib().or_sincos2pi24_batch(_p(a), _p(c), _p(s), a.size)
    return c, s


def mc_directions(seed: int, set_id: int, N: int, R: int, d: int, cell0: int = 0) -> np.ndarray:
    out = np.empty((N, R, d), np.float64)
    lib().or_mc_directions(seed, set_id, cell0, N, R, d, _p(out))
    return out


def mc_gaussians32(seed: int, set_id: int, N: int, R: int, d: int) -> np.ndarray:
    out = np.empty((N, R, d), np.float32)
    lib().or_mc_gaussians32(seed, set_id, N, R, d, _p(out))
    return out


# --- RayCast ----------------------------------------------------------------
def raycast(X, origins, dirs, eta, box: bool = True):
    """Brute-force exact RayCast of R rays; eta rows padded with NO_ID."""
    X = _f64(X)
    N, d = X.shape
    origins = _f64(origins).reshape(-1, d)
    dirs = _f64(dirs).reshape(-1, d)
    eta = np.ascontiguousarray(eta, dtype=np.int32)
    if eta.ndim == 1:
        eta = eta.reshape(-1, 1)
    R = origins.shape[0]
    hit = np.empty(R, np.int32)
    t = np.empty(R, np.float64)
    lib().or_raycast(_p(X), N, d, int(box), _p(origins), _p(dirs), _p(eta), eta.shape[1], R, _p(hit), _p(t))
    return hit, t


# --- Monte Carlo ------------------------------------------------------------
class MCResult:
    def __init__(self, hit, l, V, rowptr, col, A):
        self.hit, self.l, self.V, self.rowptr, self.col, self.A = hit, l, V, rowptr, col, A


def mc_rays(X, R: int, seed: int, set_id: int = 0):
    X = _f64(X)
    N, d = X.shape
    hit = np.empty((N, R), np.int32)
    l = np.empty((N, R), np.float64)
    lib().or_mc_rays(_p(X), N, d, R, seed, set_id, _p(hit), _p(l))
    return hit, l


def mc_reduce(X, R: int, seed: int, hit, l, set_id: int = 0):
    X = _f64(X)
    N, d = X.shape
    hit = np.ascontiguousarray(hit, dtype=np.int32)
    l = _f64(l)
    cap = N * min(R, N + 2 * d)
    V = np.empty(N)
    rowptr = np.empty(N + 1, np.int64)
    col = np.empty(cap, np.int32)
    A = np.empty(cap)
    nnz = lib().or_mc_reduce(_p(X), N, d, R, seed, set_id, _p(hit), _p(l), _p(V), _p(rowptr), _p(col), _p(A), cap)
    assert nnz >= 0
    return V, rowptr, col[:nnz].copy(), A[:nnz].copy()


def mc_integrate(X, R: int, seed: int, set_id: int = 0) -> MCResult:
    """Algorithm 3 for every cell: volumes V, CSR interface areas A."""
    hit, l = mc_rays(X, R, seed, set_id)
    V, rowptr, col, A = mc_reduce(X, R, seed, hit, l, set_id)
    return MCResult(hit, l, V, rowptr, col, A)


def mc_eval_fixed(X, R: int, seed: int, hit, rowptr, col, set_id: int = 0):
    X = _f64(X)
    N, d = X.shape
    hit = np.ascontiguousarray(hit, dtype=np.int32)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    V = np.empty(N)
    A = np.empty(col.shape[0])
    lib().or_mc_eval_fixed(_p(X), N, d, R, seed, set_id, _p(hit), _p(rowptr), _p(col), _p(V), _p(A))
    return V, A


def mc_adjoint(X, R: int, seed: int, hit, l, rowptr, col, gV, gA, set_id: int = 0):
    X = _f64(X)
    N, d = X.shape
    gX = np.empty((N, d))
    lib().or_mc_adjoint(_p(X), N, d, R, seed, set_id, _p(np.ascontiguousarray(hit, dtype=np.int32)), _p(_f64(l)),
                        _p(np.ascontiguousarray(rowptr, dtype=np.int64)), _p(np.ascontiguousarray(col, dtype=np.int32)),
                        _p(_f64(gV)), _p(_f64(gA)), _p(gX))
    return gX


# --- vertices ---------------------------------------------------------------
def vertex_coords(X, sig):
    X = _f64(X)
    sig = np.ascontiguousarray(sig, dtype=np.int32)
    r = np.empty(X.shape[1])
    ok = lib().or_vertex_coords(_p(X), X.shape[1], _p(sig), _p(r))
    return r if ok else None


def search_direction(X, sig, drop: int):
    X = _f64(X)
    sig = np.ascontiguousarray(sig, dtype=np.int32)
    u = np.empty(X.shape[1])
    ok = lib().or_search_direction(_p(X), X.shape[1], _p(sig), drop, _p(u))
    return u if ok else None


def descent(X, node: int = 0):
    X = _f64(X)
    N, d = X.shape
    sig = np.empty(d + 1, np.int32)
    ok = lib().or_descent(_p(X), N, d, node, _p(sig))
    return sig if ok else None


def vertices(X, seed_node: int = 0, max_vertices: int | None = None):
    """Algorithm 2 traversal; returns (tuples sorted lexicographically, coords, stats)."""
    X = _f64(X)
    N, d = X.shape
    if max_vertices is None:
        max_vertices = max(4096, 200 * N * (d + 1))
    tuples = np.empty((max_vertices, d + 1), np.int32)
    coords = np.empty((max_vertices, d))
    stats = np.zeros(3, np.int64)
    nv = lib().or_vertices(_p(X), N, d, seed_node, max_vertices, _p(tuples), _p(coords), _p(stats))
    if nv < 0:
        raise RuntimeError(f"oracle vertices failed: {nv}")
    tuples, coords = tuples[:nv], coords[:nv]
    order = np.lexsort(tuples.T[::-1])
    return tuples[order], coords[order], {"raycasts": int(stats[0]), "rediscoveries": int(stats[1]),
                                          "ties": int(stats[2])}


# --- Monte Carlo function integrals -------------------------------------------
def func_code(f, d: int):
    """f as (kind, axis, coef): ("one",), ("poly2", c0, b, q) or ("sin_sq", axis)."""
    coef = np.zeros(1 + 2 * d)
    if f[0] == "one":
        return 0, 0, coef
    if f[0] == "poly2":
        coef[0] = f[1]
        coef[1:1 + d] = np.asarray(f[2], dtype=np.float64)[:d]
        coef[1 + d:] = np.asarray(f[3], dtype=np.float64)[:d]
        return 1, 0, coef
    if f[0] == "sin_sq":
        return 2, int(f[1]), coef
    raise ValueError(f)


def func_eval(f, y):
    """f at the points y (n x d), by the oracle's evaluation."""
    y = _f64(np.atleast_2d(y))
    kind, axis, coef = func_code(f, y.shape[1])
    return np.array([lib().or_func_eval(kind, axis, _p(coef), y.shape[1], _p(np.ascontiguousarray(r)))
                     for r in y])


def mc_tsamples(seed: int, set_id: int, N: int, R: int, m: int) -> np.ndarray:
    """t_ks of cells 0..N-1 (N x R x m)."""
    out = np.empty((N, R, m))
    lib().or_mc_tsamples(seed, set_id, N, R, m, _p(out))
    return out


def mc_integrals(X, R: int, seed: int, cells, hit, l, rowptr, col, f, m: int, set_id: int = 0):
    """Algorithm 3's F_V (per cell) and F_d (per CSR entry) for the given
    cells: hit, l are their rows (len(cells) x R), rowptr/col their CSR rows
    (rowptr local, starting at 0).  Returns (FV, Fd)."""
    X = _f64(X)
    N, d = X.shape
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    hit = np.ascontiguousarray(hit, dtype=np.int32).reshape(len(cells), R)
    l = _f64(l).reshape(len(cells), R)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    kind, axis, coef = func_code(f, d)
    FV = np.empty(len(cells))
    Fd = np.empty(max(int(rowptr[-1]), 1))
    lib().or_mc_integrals(_p(X), N, d, R, seed, set_id, len(cells), _p(cells), _p(hit), _p(l), _p(rowptr), _p(col),
                          kind, axis, _p(coef), m, _p(FV), _p(Fd))
    return FV, Fd[:int(rowptr[-1])]


def mc_integrals_all(X, R: int, seed: int, res: MCResult, f, m: int, set_id: int = 0):
    """F_V and F_d of every cell of an oracle MC run."""
    N = X.shape[0]
    return mc_integrals(X, R, seed, np.arange(N), res.hit, res.l, res.rowptr, res.col, f, m, set_id)


def hmc(X, rowptr, col, A, tuples, coords, f):
    """Section 3.3's heuristic MC: V_H (N), F_H (nnz), I_H (N) and the vertex
    count K (nnz) of every CSR entry, from areas A and the diagram's vertices."""
    X = _f64(X)
    N, d = X.shape
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    A = _f64(A)
    tuples = np.ascontiguousarray(tuples, dtype=np.int32).reshape(-1, d + 1)
    coords = _f64(coords).reshape(-1, d)
    kind, axis, coef = func_code(f, d)
    nnz = int(rowptr[-1])
    VH, IH = np.empty(N), np.empty(N)
    FH = np.empty(max(nnz, 1))
    K = np.empty(max(nnz, 1), np.int64)
    lib().or_hmc(_p(X), N, d, _p(rowptr), _p(col), _p(A), _p(tuples), _p(coords), tuples.shape[0], kind, axis,
                 _p(coef), _p(VH), _p(FH), _p(IH), _p(K))
    return VH, FH[:nnz], IH, K[:nnz]


def leibniz(X, tuples, coords, f=("one",)):
    """Section 3.2's exact integration from the diagram's vertices: V (N), F
    (N, the integral of f's piecewise linear interpolant), and the facets'
    CSR (rowptr, col) with exact areas A and interpolant integrals Fd."""
    X = _f64(X)
    N, d = X.shape
    tuples = np.ascontiguousarray(tuples, dtype=np.int32).reshape(-1, d + 1)
    coords = _f64(coords).reshape(-1, d)
    kind, axis, coef = func_code(f, d)
    cap = 64 * N + 1024
    while True:
        V, F = np.empty(N), np.empty(N)
        rowptr = np.empty(N + 1, np.int64)
        col = np.empty(cap, np.int32)
        A, Fd = np.empty(cap), np.empty(cap)
        nnz = lib().or_leibniz(_p(X), N, d, _p(tuples), _p(coords), tuples.shape[0], kind, axis, _p(coef), _p(V),
                               _p(F), _p(rowptr), _p(col), _p(A), _p(Fd), cap)
        if nnz >= 0 or int(rowptr[-1]) <= cap:
            break
        cap = int(rowptr[-1]) + 1024
    assert nnz >= 0, "degenerate input"
    return V, F, rowptr, col[:nnz].copy(), A[:nnz].copy(), Fd[:nnz].copy()


def random_walk(X, start, steps: int, seed: int, wid=None):
    """Walkers from the vertices start (W x (d+1) sorted tuples), steps moves
    each along random edges: tuples (W x steps x (d+1)) and coordinates;
    wid: the walkers' indices in the draw (default 0..W-1)."""
    X = _f64(X)
    N, d = X.shape
    start = np.ascontiguousarray(start, dtype=np.int32).reshape(-1, d + 1)
    W = start.shape[0]
    T = np.empty((W, steps, d + 1), np.int32)
    C = np.empty((W, steps, d))
    wp = None
    if wid is not None:
        wid = np.ascontiguousarray(wid, dtype=np.int64)
        wp = _p(wid)
    rc = lib().or_random_walk(_p(X), N, d, _p(start), W, steps, seed, wp, _p(T), _p(C))
    assert rc == 0, "degenerate step"
    return T, C
