"""GPU parity of the heuristic Monte Carlo integration (Section 3.3) with the
oracle: the same areas (the GPU run's CSR) and the same vertices (the GPU
traversal's, identical to the oracle's), d = 2..5, f = 1, a positive
quadratic and sin(x_a^2).  Polynomial f: bit for bit (both sides sum in
ascending vertex order and CSR order with the same binary64 operations);
sin: within 1e-12 relative (CUDA's and libm's sin may differ in the last
bit).  f = 1 gives FH = A exactly and VH = IH = the MC volumes."""
import numpy as np
import pytest

from gpu_util import need_cuda
from paper_2405_10050_gb300 import Voronoi, synth, vd

pytestmark = pytest.mark.gpu


def _run(X, R, seed, f):
    import torch
    vor = Voronoi(X)
    mesh = vd.vd_vertices(vor.ctx)
    res = vor.mc_integrate(R, seed, keep_rays=False)
    N = X.shape[0]
    nnz = res.A.shape[0]
    VH = torch.empty(N, dtype=torch.float64, device="cuda")
    IH = torch.empty(N, dtype=torch.float64, device="cuda")
    FH = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
    vd.vd_hmc_integrals(res._mc, mesh, f, VH, FH, IH)
    nv = vd.vd_mesh_count(mesh)
    T = torch.empty((nv, X.shape[1] + 1), dtype=torch.int32, device="cuda")
    C = torch.empty((nv, X.shape[1]), dtype=torch.float64, device="cuda")
    vd.vd_mesh_copy(mesh, T, C)
    out = dict(VH=VH.cpu().numpy(), FH=FH[:nnz].cpu().numpy(), IH=IH.cpu().numpy(), V=res.V.cpu().numpy(),
               A=res.A.cpu().numpy(), rowptr=res.rowptr.cpu().numpy(), col=res.col.cpu().numpy(),
               T=T.cpu().numpy(), C=C.cpu().numpy())
    res.free()
    vd.vd_mesh_free(mesh)
    vor.close()
    return out


@pytest.mark.parametrize("d,N", [(2, 400), (3, 300), (4, 200), (5, 120)])
def test_hmc_parity(orc, d, N):
    need_cuda()
    X = synth.uniform(N, d, seed=90 + d)
    rng = np.random.default_rng(d)
    funcs = [(("one",), vd.func_one()),
             (("poly2", 0.2, list(rng.uniform(0.1, 1, d)), list(rng.uniform(0.1, 1, d))), None),
             (("sin_sq", d - 1), vd.func_sin_sq(d - 1))]
    for f, vf in funcs:
        if vf is None:
            vf = vd.func_poly2(f[1], f[2], f[3])
        g = _run(X, 128, 4, vf)
        VH, FH, IH, K = orc.hmc(X, g["rowptr"], g["col"], g["A"], g["T"], g["C"], f)
        assert np.all(K >= d)
        if f[0] == "sin_sq":
            for a, b in ((g["VH"], VH), (g["FH"], FH), (g["IH"], IH)):
                assert np.all(np.abs(a - b) <= 1e-12 * np.abs(b) + 1e-300)
        else:
            assert np.array_equal(g["VH"], VH) and np.array_equal(g["FH"], FH) and np.array_equal(g["IH"], IH)
        if f[0] == "one":
            assert np.array_equal(g["FH"], g["A"])
            assert np.all(np.abs(g["VH"] - g["V"]) <= 1e-12 * g["V"])
            assert np.all(np.abs(g["IH"] - g["VH"]) <= 1e-12 * g["VH"])


def test_hmc_host_outputs_and_errors(orc):
    need_cuda()
    X = synth.uniform(150, 3, seed=3)
    vor = Voronoi(X)
    mesh = vd.vd_vertices(vor.ctx)
    mc = vd.vd_mc_integrate(vor.ctx, 64, 2)
    try:
        N = 150
        nnz = vd.vd_mc_get(mc)
        VH, FH, IH = np.empty(N), np.empty(nnz), np.empty(N)
        vd.vd_hmc_integrals(mc, mesh, vd.func_sin_sq(0), VH, FH, IH)
        rowptr, col, A = np.empty(N + 1, np.int64), np.empty(nnz, np.int32), np.empty(nnz)
        vd.vd_mc_get(mc, rowptr=rowptr, col=col, A=A)
        nv = vd.vd_mesh_count(mesh)
        T, C = np.empty((nv, 4), np.int32), np.empty((nv, 3))
        vd.vd_mesh_copy(mesh, T, C)
        VH0, FH0, IH0, _ = orc.hmc(X, rowptr, col, A, T, C, ("sin_sq", 0))
        for a, b in ((VH, VH0), (FH, FH0), (IH, IH0)):
            assert np.all(np.abs(a - b) <= 1e-12 * np.abs(b) + 1e-300)
        IH2 = np.empty(N)
        vd.vd_hmc_integrals(mc, mesh, vd.func_one(), IH=IH2)  # only the cell integrals
        assert np.all(np.abs(IH2 - VH0) <= 1e-12 * VH0)  # f = 1: the cell integrals are the volumes
        vor2 = Voronoi(synth.uniform(100, 2, seed=1))
        mesh2 = vd.vd_vertices(vor2.ctx)
        for bad in (lambda: vd.vd_hmc_integrals(mc, mesh2, vd.func_one(), VH, FH, IH),  # d differs
                    lambda: vd.vd_hmc_integrals(mc, mesh, vd.func_sin_sq(5), VH, FH, IH),
                    lambda: vd.vd_hmc_integrals(mc, mesh, vd.func_one())):
            with pytest.raises(vd.VDError):
                bad()
        vd.vd_mesh_free(mesh2)
        vor2.close()
    finally:
        vd.vd_mc_free(mc)
        vd.vd_mesh_free(mesh)
        vor.close()


def test_voronoi_hmc_wrapper():
    """Voronoi.hmc runs the vertices, the MC areas and the heuristic rule."""
    need_cuda()
    X = synth.uniform(300, 2, seed=8)
    vor = Voronoi(X)
    VH, FH, IH, rowptr, col = vor.hmc(256, 5, vd.func_one())
    assert abs(float(VH.sum()) - 1.0) < 0.02 and float((IH - VH).abs().max()) < 1e-12
    vor.close()
