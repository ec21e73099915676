"""GPU parity of the exact integration from the vertices (Section 3.2,
Algorithms 4-5) with the oracle on the same vertices (the GPU traversal's,
identical to the oracle's): volumes, interpolant integrals, the facets' CSR,
exact areas and interface integrals for d = 2..6 and f = 1, a quadratic and
sin(x_a^2).  Both sides walk the faces in the same order with the same
binary64 operations, so polynomial f agrees bit for bit; sin within 1e-12
(CUDA's and libm's sin may differ in the last bit).  Also: the volumes tile
the unit cube, host outputs, argument errors."""
import numpy as np
import pytest

from gpu_util import need_cuda
from paper_2405_10050_gb300 import Voronoi, synth, vd

pytestmark = pytest.mark.gpu


def _gpu(X, f):
    vor = Voronoi(X)
    out = [t.cpu().numpy() for t in vor.poly(f)]
    T, C, _ = vor.vertices()
    vor.close()
    return out, T.cpu().numpy(), C.cpu().numpy()


@pytest.mark.parametrize("d,N", [(2, 300), (3, 150), (4, 60), (5, 30), (6, 12)])
def test_poly_parity(orc, d, N):
    need_cuda()
    X = synth.uniform(N, d, seed=110 + d)
    rng = np.random.default_rng(d)
    b, q = list(rng.uniform(-1, 1, d)), list(rng.uniform(0.1, 1, d))
    for f, vf in ((("one",), vd.func_one()), (("poly2", 0.4, b, q), vd.func_poly2(0.4, b, q)),
                  (("sin_sq", 0), vd.func_sin_sq(0))):
        (V, F, rp, col, A, Fd), T, C = _gpu(X, vf)
        V0, F0, rp0, col0, A0, Fd0 = orc.leibniz(X, T, C, f)
        assert np.array_equal(rp, rp0) and np.array_equal(col, col0)
        assert np.array_equal(V, V0) and np.array_equal(A, A0)
        assert abs(V.sum() - 1.0) < 1e-12
        if f[0] == "sin_sq":
            for a, r in ((F, F0), (Fd, Fd0)):
                assert np.all(np.abs(a - r) <= 1e-12 * np.abs(r) + 1e-300)
        else:
            assert np.array_equal(F, F0) and np.array_equal(Fd, Fd0)


def test_poly_host_outputs_and_errors(orc):
    need_cuda()
    X = synth.uniform(200, 3, seed=5)
    vor = Voronoi(X)
    mesh = vd.vd_vertices(vor.ctx)
    p = vd.vd_poly_integrate(vor.ctx, mesh, vd.func_poly2(1.0, [0.5, 0.25, -1.0], [0, 0, 0]))
    try:
        nnz = vd.vd_poly_get(p)
        V, F = np.empty(200), np.empty(200)
        rp, col, A, Fd = np.empty(201, np.int64), np.empty(nnz, np.int32), np.empty(nnz), np.empty(nnz)
        vd.vd_poly_get(p, V, F, rp, col, A, Fd)
        T, C, _ = vor.vertices()
        V0, F0, rp0, col0, A0, Fd0 = orc.leibniz(X, T.cpu().numpy(), C.cpu().numpy(),
                                                 ("poly2", 1.0, [0.5, 0.25, -1.0], [0, 0, 0]))
        assert np.array_equal(V, V0) and np.array_equal(F, F0) and np.array_equal(Fd, Fd0)
        for bad in (lambda: vd.vd_poly_integrate(vor.ctx, mesh, vd.func_sin_sq(3)),):
            with pytest.raises(vd.VDError):
                bad()
        vor1 = Voronoi(synth.uniform(50, 2, seed=2))
        mesh1 = vd.vd_vertices(vor1.ctx)
        with pytest.raises(vd.VDError):  # a mesh of another dimension
            vd.vd_poly_integrate(vor.ctx, mesh1, vd.func_one())
        vd.vd_mesh_free(mesh1)
        vor1.close()
    finally:
        vd.vd_poly_free(p)
        vd.vd_mesh_free(mesh)
        vor.close()


def test_poly_exact_against_mc(orc):
    """The MC volumes of Algorithm 3 scatter around the exact ones."""
    torch = need_cuda()
    X = synth.uniform(2000, 4, seed=9)
    vor = Voronoi(X)
    V = vor.poly()[0]
    res = vor.mc_integrate(1024, 3)
    S = orc.sphere_area(4)
    se = S / 4 * torch.std(res.l ** 4, dim=1) / 32.0
    z = ((res.V - V) / se).cpu().numpy()
    assert np.max(np.abs(z)) < 6.0 and abs(np.mean(z)) < 5.0 / np.sqrt(2000)
    res.free()
    vor.close()
