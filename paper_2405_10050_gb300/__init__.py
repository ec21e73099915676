"""GB300-native exact Voronoi RayCast, vertex traversal and Monte Carlo cell
integrals (Sikorski & Heida, arXiv 2405.10050).

``vd`` is the ctypes binding of the C ABI in ``include/vd.h``; ``Voronoi``
wraps a library context with torch tensors (device memory and the current
CUDA stream come from torch; all arithmetic runs in libvd's kernels), and
``VoronoiMC`` is the autograd Function of the Monte Carlo volumes and areas.
"""
from __future__ import annotations

import numpy as np

from . import vd
from .vd import NO_ID, VD_AUTO, VD_TC16, VD_FP32, VD_FP64, VDError

__all__ = ["vd", "Voronoi", "VoronoiMC", "MCResult", "NO_ID", "VD_FP64", "VD_FP32", "VD_TC16", "VD_AUTO",
           "VDError", "face_id"]


def face_id(axis: int, side: int) -> int:
    """Generator id of the box face x_axis = side (side 0 or 1)."""
    return -(2 * axis + side + 1)


class MCResult:
    """Volumes V (N), CSR areas (rowptr, col, A) and the per-ray (hit, l)."""

    def __init__(self, V, rowptr, col, A, hit=None, l=None, stats=None):
        self.V, self.rowptr, self.col, self.A, self.hit, self.l, self.stats = V, rowptr, col, A, hit, l, stats
        self._mc = None

    def adjoint(self, gV, gA):
        """gX = sum_i gV_i dV_i/dX + sum_ij gA_ij dA_ij/dX (library kernels)."""
        import torch
        N = self.V.shape[0]
        gX = torch.empty((N, self._d), dtype=torch.float64, device="cuda")
        vd.vd_mc_adjoint(self._mc, gV.to(torch.float64).contiguous(), gA.to(torch.float64).contiguous(), gX)
        return gX

    def integrals(self, f, m: int = 2):
        """Algorithm 3's function integrals of f (a vd.vd_func, e.g.
        vd.func_sin_sq(0)): F_V per cell (N) and F_d per CSR entry (aligned
        with col), m samples along each ray for F_V (library kernels)."""
        import torch
        FV = torch.empty(self.V.shape[0], dtype=torch.float64, device="cuda")
        Fd = torch.empty(max(self.A.shape[0], 1), dtype=torch.float64, device="cuda")
        vd.vd_mc_integrals(self._mc, f, m, FV, Fd)
        return FV, Fd[:self.A.shape[0]]

    def free(self):
        if self._mc is not None:
            vd.vd_mc_free(self._mc)
            self._mc = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Voronoi:
    """A libvd context holding one node set X (N x d, float64)."""

    def __init__(self, X, precision: int = VD_AUTO, box: bool = True, stream=None, knn_k: int = 0):
        """knn_k: candidate list length per node (0 automatic, -1 tree walk only)."""
        import torch
        cfg = vd.vd_config_default()
        cfg.precision = precision
        cfg.box = int(box)
        cfg.knn_k = knn_k
        self._stream = stream
        self.ctx = vd.vd_create(cfg, stream)
        self.X = None
        self.set_nodes(X)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            vd.vd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_nodes(self, X):
        import torch
        if not torch.is_tensor(X):
            X = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float64))
        X = X.to(device="cuda", dtype=torch.float64).contiguous()
        vd.vd_set_nodes(self.ctx, X)
        self.X = X
        self.N, self.d = X.shape

    def set_precision(self, precision: int):
        vd.vd_set_precision(self.ctx, precision)

    def stats(self):
        return vd.vd_last_stats(self.ctx)

    def raycast(self, origins, dirs, eta, screen_err: bool = False):
        """Exact first hit of each ray; eta rows start with the reference node."""
        import torch
        dev = torch.device("cuda")
        origins = torch.as_tensor(origins, dtype=torch.float64, device=dev).contiguous()
        dirs = torch.as_tensor(dirs, dtype=torch.float64, device=dev).contiguous()
        eta = torch.as_tensor(eta, dtype=torch.int32, device=dev)
        if eta.dim() == 1:
            eta = eta[:, None]
        eta = eta.contiguous()
        R = origins.shape[0]
        hit = torch.empty(R, dtype=torch.int32, device=dev)
        t = torch.empty(R, dtype=torch.float64, device=dev)
        se = torch.empty(R, dtype=torch.float32, device=dev) if screen_err else None
        vd.vd_raycast(self.ctx, origins, dirs, eta, hit, t, se)
        return (hit, t, se) if screen_err else (hit, t)

    def directions(self, seed: int, ncells: int, R: int, cell0: int = 0, set_id: int = 0):
        import torch
        out = torch.empty((ncells, R, self.d), dtype=torch.float64, device="cuda")
        vd.vd_mc_directions(self.ctx, seed, set_id, cell0, ncells, R, self.d, out)
        return out

    def mc_integrate(self, rays_per_cell: int, seed: int, keep_rays: bool = True) -> MCResult:
        import torch
        mc = vd.vd_mc_integrate(self.ctx, rays_per_cell, seed)
        try:
            N = self.N
            V = torch.empty(N, dtype=torch.float64, device="cuda")
            rowptr = torch.empty(N + 1, dtype=torch.int64, device="cuda")
            nnz = vd.vd_mc_get(mc, V=V, rowptr=rowptr)
            col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
            A = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
            vd.vd_mc_get(mc, col=col, A=A)
            hit = l = None
            if keep_rays:
                hit = torch.empty((N, rays_per_cell), dtype=torch.int32, device="cuda")
                l = torch.empty((N, rays_per_cell), dtype=torch.float64, device="cuda")
                vd.vd_mc_rays(mc, hit, l)
            res = MCResult(V, rowptr, col[:nnz], A[:nnz], hit, l, vd.vd_mc_stats(mc))
            res._mc = mc
            res._d = self.d
            mc = None
            return res
        finally:
            if mc is not None:
                vd.vd_mc_free(mc)

    def hmc(self, rays_per_cell: int, seed: int, f):
        """Heuristic MC (Section 3.3) of f (a vd.vd_func): the MC areas with
        rays_per_cell rays, the vertices of the diagram, then the volumes VH,
        interface integrals FH (CSR: rowptr, col) and cell integrals IH."""
        import torch
        mesh = vd.vd_vertices(self.ctx)
        try:
            res = self.mc_integrate(rays_per_cell, seed, keep_rays=False)
            try:
                N = self.N
                VH = torch.empty(N, dtype=torch.float64, device="cuda")
                IH = torch.empty(N, dtype=torch.float64, device="cuda")
                FH = torch.empty(max(res.A.shape[0], 1), dtype=torch.float64, device="cuda")
                vd.vd_hmc_integrals(res._mc, mesh, f, VH, FH, IH)
                return VH, FH[:res.A.shape[0]], IH, res.rowptr, res.col
            finally:
                res.free()
        finally:
            vd.vd_mesh_free(mesh)

    def poly(self, f=None):
        """Exact integration from the vertices (Section 3.2): volumes V,
        integrals F of f's piecewise linear interpolant, the facets' CSR
        (rowptr, col) with exact areas A and interface integrals Fd."""
        import torch
        f = f if f is not None else vd.func_one()
        mesh = vd.vd_vertices(self.ctx)
        try:
            p = vd.vd_poly_integrate(self.ctx, mesh, f)
        finally:
            vd.vd_mesh_free(mesh)
        try:
            N = self.N
            nnz = vd.vd_poly_get(p)
            dev = dict(device="cuda")
            V, F = torch.empty(N, dtype=torch.float64, **dev), torch.empty(N, dtype=torch.float64, **dev)
            rowptr = torch.empty(N + 1, dtype=torch.int64, **dev)
            col = torch.empty(max(nnz, 1), dtype=torch.int32, **dev)
            A = torch.empty(max(nnz, 1), dtype=torch.float64, **dev)
            Fd = torch.empty(max(nnz, 1), dtype=torch.float64, **dev)
            vd.vd_poly_get(p, V, F, rowptr, col, A, Fd)
            return V, F, rowptr, col[:nnz], A[:nnz], Fd[:nnz]
        finally:
            vd.vd_poly_free(p)

    def random_walk(self, start, steps: int, seed: int):
        """Walkers from the vertices start (W x (d+1) sorted tuples, e.g. rows
        of vertices()), steps random edges each (Section 2.3): the visited
        tuples (W x steps x (d+1)) and coordinates."""
        import torch
        start = torch.as_tensor(start, dtype=torch.int32, device="cuda").contiguous()
        W = start.shape[0]
        T = torch.empty((W, steps, self.d + 1), dtype=torch.int32, device="cuda")
        C = torch.empty((W, steps, self.d), dtype=torch.float64, device="cuda")
        vd.vd_random_walk(self.ctx, start, steps, seed, T, C)
        return T, C

    def vertices(self, cells_per_batch=None):
        """All vertices of the clipped diagram: (tuples V x (d+1), coords V x d,
        stats).  cells_per_batch: None for the whole-diagram traversal, else the
        per-cell exploration in batches of that many cells (0 = automatic)."""
        import torch
        m = vd.vd_vertices(self.ctx) if cells_per_batch is None else vd.vd_vertices_by_cells(self.ctx, cells_per_batch)
        try:
            nv = vd.vd_mesh_count(m)
            tuples = torch.empty((nv, self.d + 1), dtype=torch.int32, device="cuda")
            coords = torch.empty((nv, self.d), dtype=torch.float64, device="cuda")
            if nv:
                vd.vd_mesh_copy(m, tuples, coords)
            return tuples, coords, vd.vd_mesh_stats(m)
        finally:
            vd.vd_mesh_free(m)


class VoronoiMC:
    """torch.autograd.Function: X -> (V, A, rowptr, col) by Algorithm 3; V
    and A are differentiable, backward runs the library's adjoint kernels on
    the saved per-ray argmins (directions fixed, pathwise)."""

    @staticmethod
    def apply(X, rays_per_cell: int, seed: int, precision: int = VD_AUTO):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx_, Xin):
                vor = Voronoi(Xin.detach(), precision=precision)
                res = vor.mc_integrate(rays_per_cell, seed, keep_rays=False)
                ctx_.res = res
                ctx_.vor = vor
                ctx_.mark_non_differentiable(res.rowptr, res.col)
                return res.V.clone(), res.A.clone(), res.rowptr, res.col

            @staticmethod
            def backward(ctx_, gV, gA, _g_rowptr=None, _g_col=None):
                res = ctx_.res
                gV = gV if gV is not None else torch.zeros_like(res.V)
                gA = gA if gA is not None else torch.zeros_like(res.A)
                return res.adjoint(gV, gA)

        return _Fn.apply(X)
