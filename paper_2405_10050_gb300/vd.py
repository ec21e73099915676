"""ctypes binding of libvd (include/vd.h).

The functions keep the C names and only marshal arguments: arrays may be
CUDA torch tensors (passed as device pointers) or numpy arrays / CPU tensors
(passed as host pointers); every computation runs in the library's CUDA
kernels.  The library must have been built (``paper_2405_10050_gb300.build``):
loading fails loudly otherwise, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

NO_ID = -(2**31)
VD_FP64, VD_FP32, VD_TC16, VD_AUTO = 0, 1, 2, 3
STATUS = {0: "VD_OK", -1: "VD_EINVAL", -2: "VD_ENOMEM", -3: "VD_ECUDA", -4: "VD_EDEGENERATE",
          -5: "VD_EHASHFULL", -6: "VD_EOVERFLOW", -7: "VD_ETIMEOUT"}


class VDError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class vd_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("box", ctypes.c_int32), ("hash_capacity", ctypes.c_int64),
                ("max_levels", ctypes.c_int64), ("wait_limit", ctypes.c_int64), ("knn_k", ctypes.c_int32),
                ("rays_per_block", ctypes.c_int32)]


VD_F_ONE, VD_F_POLY2, VD_F_SIN_SQ = 0, 1, 2


class vd_func(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("axis", ctypes.c_int32), ("c0", ctypes.c_double),
                ("b", ctypes.c_double * 16), ("q", ctypes.c_double * 16)]


def func_one():
    """f = 1."""
    return vd_func(kind=VD_F_ONE)


def func_poly2(c0, b=(), q=()):
    """f = c0 + sum_a b[a] y_a + sum_a q[a] y_a^2."""
    f = vd_func(kind=VD_F_POLY2, c0=float(c0))
    for a, v in enumerate(b):
        f.b[a] = float(v)
    for a, v in enumerate(q):
        f.q[a] = float(v)
    return f


def func_sin_sq(axis=0):
    """f = sin(y_axis^2)."""
    return vd_func(kind=VD_F_SIN_SQ, axis=int(axis))


class vd_stats(ctypes.Structure):
    _fields_ = [("rays", ctypes.c_int64), ("tiles_visited", ctypes.c_int64), ("pairs_screened", ctypes.c_int64),
                ("rechecked", ctypes.c_int64), ("fallback_rays", ctypes.c_int64), ("overflow_rays", ctypes.c_int64),
                ("ties", ctypes.c_int64), ("levels", ctypes.c_int64), ("vertices", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("raycast_ms", ctypes.c_double),
                ("edge_table_bytes", ctypes.c_int64), ("vertex_table_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["vd_kernel_launches", "vd_config_default", "vd_create", "vd_destroy", "vd_last_error", "vd_status_str", "vd_set_precision",
           "vd_last_stats", "vd_set_nodes", "vd_raycast", "vd_vertices", "vd_vertices_by_cells", "vd_mesh_count", "vd_mesh_dim",
           "vd_mesh_copy", "vd_mesh_stats", "vd_mesh_free", "vd_mc_integrate", "vd_mc_get", "vd_mc_rays",
           "vd_mc_adjoint", "vd_mc_integrals", "vd_hmc_integrals", "vd_mc_stats", "vd_mc_count", "vd_mc_free", "vd_mc_directions",
           "vd_mc_integrate_batch", "vd_raycast_noalloc", "vd_poly_integrate", "vd_poly_get", "vd_poly_free", "vd_random_walk"]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libvd.so (building it first when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libvd.so is not built; run paper_2405_10050_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    P, i32, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "vd_kernel_launches": (i64, []),
        "vd_config_default": (None, [P]),
        "vd_create": (i32, [P, P, P]),
        "vd_destroy": (None, [P]),
        "vd_last_error": (ctypes.c_char_p, [P]),
        "vd_status_str": (ctypes.c_char_p, [i32]),
        "vd_set_precision": (i32, [P, i32]),
        "vd_last_stats": (i32, [P, P]),
        "vd_set_nodes": (i32, [P, P, i64, i32, i32]),
        "vd_raycast": (i32, [P, P, P, P, i32, i64, P, P, P, i32]),
        "vd_raycast_noalloc": (i32, [P, P, P, P, i32, i64, P, P]),
        "vd_vertices": (i32, [P, P]),
        "vd_vertices_by_cells": (i32, [P, i64, P]),
        "vd_mesh_count": (i64, [P]),
        "vd_mesh_dim": (i32, [P]),
        "vd_mesh_copy": (i32, [P, P, P, i32]),
        "vd_mesh_stats": (i32, [P, P]),
        "vd_mesh_free": (None, [P]),
        "vd_mc_integrate": (i32, [P, i64, u64, P]),
        "vd_mc_get": (i32, [P, P, P, P, P, P, i32]),
        "vd_mc_rays": (i32, [P, P, P, i32]),
        "vd_mc_adjoint": (i32, [P, P, P, P, i32]),
        "vd_mc_integrals": (i32, [P, P, i64, P, P, i32]),
        "vd_hmc_integrals": (i32, [P, P, P, P, P, P, i32]),
        "vd_poly_integrate": (i32, [P, P, P, P]),
        "vd_poly_get": (i32, [P, P, P, P, P, P, P, P, i32]),
        "vd_poly_free": (None, [P]),
        "vd_random_walk": (i32, [P, P, i64, i64, u64, P, P, i32]),
        "vd_mc_stats": (i32, [P, P]),
        "vd_mc_count": (i64, [P]),
        "vd_mc_free": (None, [P]),
        "vd_mc_directions": (i32, [P, u64, u32, i64, i64, i64, i32, P, i32]),
        "vd_mc_integrate_batch": (i32, [P, i32, P, P, P, i64, u64, P, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# ---------------------------------------------------------------- helpers --
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, on_device, keepalive) for a torch tensor or numpy array."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32,
               np.int64: torch.int64}[dtype]
        assert a.dtype == tdt and a.is_contiguous(), f"expected contiguous {tdt}"
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


def _check(ctx, st):
    if st != 0:
        msg = load().vd_last_error(ctx).decode() if ctx else ""
        raise VDError(st, msg)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(int(stream))


# ----------------------------------------------------------- thin wrappers --
def vd_kernel_launches():
    return int(load().vd_kernel_launches())


def vd_config_default():
    cfg = vd_config()
    load().vd_config_default(ctypes.byref(cfg))
    return cfg


def vd_create(cfg=None, stream=None):
    L = load()
    ctx = ctypes.c_void_p()
    st = L.vd_create(ctypes.byref(ctx), ctypes.byref(cfg) if cfg is not None else None, _stream_ptr(stream))
    _check(None, st)
    return ctx


def vd_destroy(ctx):
    load().vd_destroy(ctx)


def vd_set_precision(ctx, precision):
    _check(ctx, load().vd_set_precision(ctx, int(precision)))


def vd_last_stats(ctx):
    s = vd_stats()
    _check(ctx, load().vd_last_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def vd_set_nodes(ctx, X):
    p, dev, keep = _ptr(X, np.float64)
    N, d = X.shape
    _check(ctx, load().vd_set_nodes(ctx, p, N, d, dev))


def vd_raycast(ctx, origins, dirs, eta, hit, t, screen_err=None):
    po, dev, k1 = _ptr(origins, np.float64)
    pu, _, k2 = _ptr(dirs, np.float64)
    pe, _, k3 = _ptr(eta, np.int32)
    ph, _, k4 = _ptr(hit, np.int32)
    pt, _, k5 = _ptr(t, np.float64)
    ps, _, k6 = _ptr(screen_err, np.float32)
    R = origins.shape[0]
    stride = eta.shape[1] if len(eta.shape) == 2 else 1
    _check(ctx, load().vd_raycast(ctx, po, pu, pe, stride, R, ph, pt, ps, dev))
    if not dev:  # numpy outputs were copied into contiguous buffers
        if k4 is not hit:
            hit[...] = k4
        if k5 is not t:
            t[...] = k5
        if screen_err is not None and k6 is not screen_err:
            screen_err[...] = k6


def vd_raycast_noalloc(ctx, origins, dirs, eta, hit, t):
    """Allocation-free RayCast: all arrays must be CUDA tensors."""
    args = [_ptr(a, dt) for a, dt in ((origins, np.float64), (dirs, np.float64), (eta, np.int32),
                                      (hit, np.int32), (t, np.float64))]
    if any(a[1] != 1 for a in args):
        raise ValueError("vd_raycast_noalloc takes device (CUDA) arrays only")
    stride = eta.shape[1] if len(eta.shape) == 2 else 1
    _check(ctx, load().vd_raycast_noalloc(ctx, args[0][0], args[1][0], args[2][0], stride, origins.shape[0],
                                          args[3][0], args[4][0]))


def vd_mc_directions(ctx, seed, set_id, cell0, ncells, R, d, out):
    p, dev, keep = _ptr(out, np.float64)
    _check(ctx, load().vd_mc_directions(ctx, seed, set_id, cell0, ncells, R, d, p, dev))
    if not dev and keep is not out:
        out[...] = keep


def vd_mc_integrate(ctx, rays_per_cell, seed):
    mc = ctypes.c_void_p()
    _check(ctx, load().vd_mc_integrate(ctx, rays_per_cell, seed, ctypes.byref(mc)))
    return mc


def vd_mc_get(mc, V=None, rowptr=None, col=None, A=None):
    nnz = ctypes.c_int64()
    args = [_ptr(V, np.float64), _ptr(rowptr, np.int64), _ptr(col, np.int32), _ptr(A, np.float64)]
    dev = next((a[1] for a in args if a[1] is not None), 0)
    st = load().vd_mc_get(mc, args[0][0], ctypes.byref(nnz), args[1][0], args[2][0], args[3][0], dev)
    _check(None, st)
    return nnz.value


def vd_mc_integrate_batch(ctx, Xs, rays_per_cell, seed):
    """Batched MC over a list of node sets (torch CUDA tensors or numpy
    arrays, all of one kind); returns one vd_mc handle per set."""
    ptrs, keep, dev = [], [], None
    for X in Xs:
        p, dv, k = _ptr(X, np.float64)
        if dev is None:
            dev = dv
        elif dev != dv:
            raise ValueError("all sets must be on the same side (host or device)")
        ptrs.append(p.value)
        keep.append(k)
    n = len(Xs)
    Pa = (ctypes.c_void_p * n)(*ptrs)
    Na = (ctypes.c_int64 * n)(*[X.shape[0] for X in Xs])
    Da = (ctypes.c_int32 * n)(*[X.shape[1] for X in Xs])
    outs = (ctypes.c_void_p * n)()
    _check(ctx, load().vd_mc_integrate_batch(ctx, n, Pa, Na, Da, rays_per_cell, seed, outs, dev or 0))
    return [ctypes.c_void_p(o) for o in outs]


def vd_mc_rays(mc, hit, l):
    ph, dev, _ = _ptr(hit, np.int32)
    pl, _, _ = _ptr(l, np.float64)
    _check(None, load().vd_mc_rays(mc, ph, pl, dev))


def vd_mc_adjoint(mc, gV, gA, gX):
    pv, dev, k1 = _ptr(gV, np.float64)
    pa, dev2, k2 = _ptr(gA, np.float64)
    px, dev3, k3 = _ptr(gX, np.float64)
    _check(None, load().vd_mc_adjoint(mc, pv, pa, px, dev3))


def vd_mc_integrals(mc, f, m, FV=None, Fd=None):
    """Algorithm 3's F_V (N) and F_d (nnz, vd_mc_get's col order) of f
    (a vd_func) with m samples per ray."""
    pv, dev, k1 = _ptr(FV, np.float64)
    pd, dev2, k2 = _ptr(Fd, np.float64)
    dev = dev if dev is not None else (dev2 or 0)
    _check(None, load().vd_mc_integrals(mc, ctypes.byref(f), int(m), pv, pd, dev))


def vd_hmc_integrals(mc, mesh, f, VH=None, FH=None, IH=None):
    """Section 3.3's heuristic MC: VH (N), FH (nnz, vd_mc_get's col order),
    IH (N) from the areas of mc and the vertices of mesh."""
    ptrs = [_ptr(VH, np.float64), _ptr(FH, np.float64), _ptr(IH, np.float64)]
    dev = next((p[1] for p in ptrs if p[1] is not None), 0)
    _check(None, load().vd_hmc_integrals(mc, mesh, ctypes.byref(f), ptrs[0][0], ptrs[1][0], ptrs[2][0], dev))


def vd_poly_integrate(ctx, mesh, f):
    """Section 3.2's exact integration of the context's nodes from mesh."""
    p = ctypes.c_void_p()
    _check(ctx, load().vd_poly_integrate(ctx, mesh, ctypes.byref(f), ctypes.byref(p)))
    return p


def vd_poly_get(p, V=None, F=None, rowptr=None, col=None, A=None, Fd=None):
    nnz = ctypes.c_int64()
    args = [_ptr(V, np.float64), _ptr(F, np.float64), _ptr(rowptr, np.int64), _ptr(col, np.int32),
            _ptr(A, np.float64), _ptr(Fd, np.float64)]
    dev = next((a[1] for a in args if a[1] is not None), 0)
    _check(None, load().vd_poly_get(p, args[0][0], args[1][0], ctypes.byref(nnz), args[2][0], args[3][0], args[4][0],
                                    args[5][0], dev))
    return nnz.value


def vd_poly_free(p):
    load().vd_poly_free(p)


def vd_random_walk(ctx, start, steps, seed, path_tuples, path_coords=None):
    """W walkers from the vertices start (W x (d+1)), steps moves each."""
    ps, dev, k1 = _ptr(start, np.int32)
    pt, dev2, k2 = _ptr(path_tuples, np.int32)
    pc, dev3, k3 = _ptr(path_coords, np.float64)
    W = int(start.shape[0])
    _check(ctx, load().vd_random_walk(ctx, ps, W, int(steps), int(seed), pt, pc, dev or 0))


def vd_mc_stats(mc):
    s = vd_stats()
    _check(None, load().vd_mc_stats(mc, ctypes.byref(s)))
    return s.as_dict()


def vd_mc_count(mc):
    return int(load().vd_mc_count(mc))


def vd_mc_free(mc):
    load().vd_mc_free(mc)


def vd_vertices(ctx):
    m = ctypes.c_void_p()
    _check(ctx, load().vd_vertices(ctx, ctypes.byref(m)))
    return m


def vd_vertices_by_cells(ctx, cells_per_batch: int = 0):
    m = ctypes.c_void_p()
    _check(ctx, load().vd_vertices_by_cells(ctx, int(cells_per_batch), ctypes.byref(m)))
    return m


def vd_mesh_count(mesh):
    return int(load().vd_mesh_count(mesh))


def vd_mesh_dim(mesh):
    return int(load().vd_mesh_dim(mesh))


def vd_mesh_copy(mesh, tuples=None, coords=None):
    pt, dev, _ = _ptr(tuples, np.int32)
    pc, dev2, _ = _ptr(coords, np.float64)
    dev = dev if dev is not None else (dev2 or 0)
    _check(None, load().vd_mesh_copy(mesh, pt, pc, dev))


def vd_mesh_stats(mesh):
    s = vd_stats()
    _check(None, load().vd_mesh_stats(mesh, ctypes.byref(s)))
    return s.as_dict()


def vd_mesh_free(mesh):
    load().vd_mesh_free(mesh)
