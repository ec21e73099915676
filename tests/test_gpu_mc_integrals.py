"""GPU parity of the Monte Carlo function integrals (Section 3.1, Algorithm
3's F_d and F_V) with the oracle, on the same rays: f = 1, a positive
quadratic and sin(x_a^2), d = 1..16, m = 1..5 samples per ray, both orders
of the facet sums (many and few rays per facet), host and device outputs,
batched sets; F_d(f = 1) equals the library's own A bit for bit, and runs
that keep the directions and runs that draw them again agree bit for bit.
Sums are compared within 1e-12 relative (every term is positive, and the GPU
adds them in another fixed order)."""
import numpy as np
import pytest

from gpu_util import need_cuda
from paper_2405_10050_gb300 import VD_FP32, VD_FP64, Voronoi, synth, vd

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(8)
B = list(RNG.uniform(0.1, 1.0, 16))
Q = list(RNG.uniform(0.1, 1.0, 16))


def _funcs(d):
    return [("one",), ("poly2", 0.3, B, Q), ("sin_sq", d - 1)]


def _vdf(f):
    if f[0] == "one":
        return vd.func_one()
    if f[0] == "poly2":
        return vd.func_poly2(f[1], f[2], f[3])
    return vd.func_sin_sq(f[1])


def _close(a, b, rel=1e-12):
    a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
    assert a.shape == b.shape
    assert np.all(np.abs(a - b) <= rel * np.abs(b) + 1e-300), np.max(np.abs(a - b) / (np.abs(b) + 1e-300))


def _oracle(orc, X, R, seed, res, f, m, set_id=0):
    N = X.shape[0]
    return orc.mc_integrals(X, R, seed, np.arange(N), res.hit.cpu().numpy(), res.l.cpu().numpy(),
                            res.rowptr.cpu().numpy(), res.col.cpu().numpy(), f, m, set_id)


@pytest.mark.parametrize("d,N,R,m", [(1, 50, 64, 3), (2, 300, 256, 2), (3, 500, 128, 5), (4, 400, 64, 4),
                                     (5, 300, 64, 1), (8, 200, 48, 2), (12, 150, 32, 3), (16, 120, 32, 2)])
def test_integrals_parity(orc, d, N, R, m):
    torch = need_cuda()
    X = synth.uniform(N, d, seed=60 + d)
    vor = Voronoi(X)
    res = vor.mc_integrate(R, 5)
    for f in _funcs(d):
        FV, Fd = res.integrals(_vdf(f), m)
        FV0, Fd0 = _oracle(orc, X, R, 5, res, f, m)
        _close(FV, FV0)
        _close(Fd, Fd0)
        if f[0] == "one":
            assert torch.equal(Fd, res.A)
    res.free()
    vor.close()


def test_few_rays_per_facet_order(orc):
    """High d with few rays: (almost) every row takes the ray-parallel order
    of the facet sums (nnz * 8 > R)."""
    torch = need_cuda()
    X = synth.gaussian_mixture(400, 10, K=4, sigma=0.1, seed=3)
    vor = Voronoi(X)
    res = vor.mc_integrate(16, 2)
    nnz_row = np.diff(res.rowptr.cpu().numpy())
    assert np.mean(nnz_row * 8 > 16) > 0.9
    for f in _funcs(10):
        FV, Fd = res.integrals(_vdf(f), 3)
        FV0, Fd0 = _oracle(orc, X, 16, 2, res, f, 3)
        _close(FV, FV0)
        _close(Fd, Fd0)
        if f[0] == "one":
            assert torch.equal(Fd, res.A)
    res.free()
    vor.close()


def test_kept_and_redrawn_directions_agree():
    """The candidate-list kernels keep each ray's direction for the later
    passes; the binary64 path draws it again: the integrals are identical."""
    torch = need_cuda()
    X = synth.uniform(600, 3, seed=5)
    out = []
    for prec in (VD_FP32, VD_FP64):
        vor = Voronoi(X, precision=prec)
        res = vor.mc_integrate(64, 9)
        out.append([t.clone() for t in res.integrals(vd.func_sin_sq(1), 3)])
        res.free()
        vor.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_host_outputs_and_errors(orc):
    need_cuda()
    X = synth.uniform(200, 2, seed=4)
    vor = Voronoi(X)
    mc = vd.vd_mc_integrate(vor.ctx, 32, 1)
    try:
        N = 200
        nnz = vd.vd_mc_get(mc)
        FV = np.empty(N)
        Fd = np.empty(nnz)
        vd.vd_mc_integrals(mc, vd.func_poly2(0.5, [1.0, 2.0], [0.5, 0.25]), 2, FV, Fd)
        hit = np.empty((N, 32), np.int32)
        l = np.empty((N, 32))
        vd.vd_mc_rays(mc, hit, l)
        rowptr = np.empty(N + 1, np.int64)
        col = np.empty(nnz, np.int32)
        vd.vd_mc_get(mc, rowptr=rowptr, col=col)
        f = ("poly2", 0.5, [1.0, 2.0], [0.5, 0.25])
        FV0, Fd0 = orc.mc_integrals(X, 32, 1, np.arange(N), hit, l, rowptr, col, f, 2)
        _close(FV, FV0)
        _close(Fd, Fd0)
        FV2 = np.empty(N)
        vd.vd_mc_integrals(mc, vd.func_one(), 1, FV=FV2)  # F_d not asked for
        assert np.all(FV2 > 0)
        for bad in (lambda: vd.vd_mc_integrals(mc, vd.func_sin_sq(2), 1, FV, Fd),  # axis >= d
                    lambda: vd.vd_mc_integrals(mc, vd.func_one(), 0, FV, Fd),      # m < 1
                    lambda: vd.vd_mc_integrals(mc, vd.vd_func(kind=7), 1, FV, Fd),
                    lambda: vd.vd_mc_integrals(mc, vd.func_one(), 1)):
            with pytest.raises(vd.VDError):
                bad()
    finally:
        vd.vd_mc_free(mc)
        vor.close()


def test_batched_sets(orc):
    """Integrals of sets of a batched run use the set's Philox set id."""
    torch = need_cuda()
    sets = synth.batch_sets(6, seed=2)
    ctx = vd.vd_create(None, torch.cuda.current_stream().cuda_stream)
    try:
        Xd = [torch.tensor(X, device="cuda") for X, _ in sets]
        mcs = vd.vd_mc_integrate_batch(ctx, Xd, 64, 3)
        for s in (0, 3, 5):
            X = sets[s][0]
            N, d = X.shape
            nnz = vd.vd_mc_get(mcs[s])
            rowptr = np.empty(N + 1, np.int64)
            col = np.empty(nnz, np.int32)
            vd.vd_mc_get(mcs[s], rowptr=rowptr, col=col)
            hit = np.empty((N, 64), np.int32)
            l = np.empty((N, 64))
            vd.vd_mc_rays(mcs[s], hit, l)
            f = ("sin_sq", 0)
            FV = np.empty(N)
            Fd = np.empty(nnz)
            vd.vd_mc_integrals(mcs[s], vd.func_sin_sq(0), 2, FV, Fd)
            FV0, Fd0 = orc.mc_integrals(X, 64, 3, np.arange(N), hit, l, rowptr, col, f, 2, set_id=s)
            _close(FV, FV0)
            _close(Fd, Fd0)
        for mc in mcs:
            vd.vd_mc_free(mc)
    finally:
        vd.vd_destroy(ctx)
