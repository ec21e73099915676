"""GPU parity of the Monte Carlo integrals (Section 3.1, Algorithm 3) and of
their adjoint against the FP64 oracle on the same seeded directions."""
import numpy as np
import pytest

from gpu_util import need_cuda
from paper_2405_10050_gb300 import VD_FP32, VD_FP64, VD_TC16, Voronoi, VoronoiMC, synth, vd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d", list(range(1, 17)))
def test_directions_bitwise(orc, d):
    """The GPU draw (Philox4x32-10, binary32 Box-Muller with series-defined
    log/sin/cos, binary64 normalisation) equals the oracle's bit for bit."""
    need_cuda()
    vor = Voronoi(synth.uniform(4, d, seed=0))
    for seed, set_id, cell0 in [(0, 0, 0), (12345, 3, 1000), (2**63 + 17, 511, 2**31 + 5)]:
        g = vor.directions(seed, 40, 37, cell0=cell0, set_id=set_id).cpu().numpy()
        ref = orc.mc_directions(seed, set_id, 40, 37, d, cell0=cell0)
        assert np.array_equal(g, ref)
    vor.close()


def _parity(orc, X, R, seed, prec, knn_k=0):
    vor = Voronoi(X, precision=prec, knn_k=knn_k)
    res = vor.mc_integrate(R, seed)
    ref = orc.mc_integrate(X, R, seed)
    hit, l = res.hit.cpu().numpy(), res.l.cpu().numpy()
    assert np.array_equal(hit, ref.hit)
    assert np.array_equal(l, ref.l)
    V = res.V.cpu().numpy()
    assert np.allclose(V, ref.V, rtol=1e-12, atol=0)
    assert np.array_equal(res.rowptr.cpu().numpy(), ref.rowptr)
    assert np.array_equal(res.col.cpu().numpy(), ref.col)
    assert np.allclose(res.A.cpu().numpy(), ref.A, rtol=1e-12, atol=0)
    return vor, res, ref


@pytest.mark.parametrize("prec", [VD_FP64, VD_FP32, VD_TC16])
@pytest.mark.parametrize("d,N,R", [(1, 100, 16), (2, 700, 64), (3, 2000, 64), (4, 1000, 64), (5, 600, 32),
                                   (8, 300, 32), (16, 200, 16)])
def test_mc_parity(orc, prec, d, N, R):
    need_cuda()
    X = synth.uniform(N, d, seed=d)
    vor, res, ref = _parity(orc, X, R, seed=11 + d, prec=prec)
    res.free()
    vor.close()


@pytest.mark.parametrize("d,N,R,scale", [(3, 3000, 200, 1.0), (4, 1500, 130, 1e-3), (6, 800, 96, 1.0),
                                         (12, 300, 40, 1.0)])
def test_mc_parity_tensor_cases(orc, d, N, R, scale):
    """Tensor-core screening: clustered nodes, several 128-ray tiles per
    cell with a ragged last tile (R not a multiple of 128), and a small-scale
    set whose offsets fall below the fp16 normal range (the absolute error
    floor of the bound)."""
    need_cuda()
    X = synth.gaussian_mixture(N, d, K=8, sigma=0.03, seed=d) * scale
    vor, res, ref = _parity(orc, X, R, seed=7 + d, prec=VD_TC16)
    res.free()
    vor.close()


@pytest.mark.parametrize("d,N,R,mix", [(3, 1500, 64, False), (5, 700, 32, True), (9, 400, 96, False),
                                       (12, 300, 200, True), (16, 500, 64, True), (16, 33, 128, False)])
def test_mc_parity_tensor_walk(orc, d, N, R, mix):
    """Block tree walk with tensor-core ball tests and leaf screening (the
    path of node sets without candidate lists): 1, 2 and 4 cells per ray
    tile (R = 96 or 200, 64, 32), ragged last tiles, a set of one tile and
    one more node."""
    need_cuda()
    X = synth.gaussian_mixture(N, d, K=4, sigma=0.1, seed=d) if mix else synth.uniform(N, d, seed=d)
    vor, res, ref = _parity(orc, X, R, seed=21 + d, prec=VD_TC16, knn_k=-1)
    assert res.stats["tiles_visited"] > 0
    res.free()
    vor.close()


@pytest.mark.parametrize("d,N,R", [(2, 300, 32), (3, 300, 32), (4, 300, 32), (2, 200, 512), (3, 150, 256),
                                   (9, 120, 16), (4, 120, 1100)])
def test_adjoint_parity(orc, d, N, R):
    """Rows with many rays per hit id (R = 256, 512, 1100: rays sorted by entry,
    R = 1100 in several chunks with a ragged last one) and rows with few
    (R = 16, 32: 32 rays at a time, summed per entry)."""
    torch = need_cuda()
    X = synth.uniform(N, d, seed=50 + d)
    vor, res, ref = _parity(orc, X, R, seed=3, prec=VD_FP32)
    rng = np.random.default_rng(d)
    gV = rng.standard_normal(N)
    gA = rng.standard_normal(ref.col.shape[0])
    gX = res.adjoint(torch.tensor(gV, device="cuda"), torch.tensor(gA, device="cuda")).cpu().numpy()
    gX0 = orc.mc_adjoint(X, R, 3, ref.hit, ref.l, ref.rowptr, ref.col, gV, gA)
    assert np.max(np.abs(gX - gX0)) <= 1e-10 * np.max(np.abs(gX0))
    # deterministic: a second call gives identical bits
    gX2 = res.adjoint(torch.tensor(gV, device="cuda"), torch.tensor(gA, device="cuda")).cpu().numpy()
    assert np.array_equal(gX, gX2)
    res.free()
    vor.close()


def test_autograd_function(orc):
    torch = need_cuda()
    N, R, d = 200, 32, 3
    X = torch.tensor(synth.uniform(N, d, seed=9), device="cuda", requires_grad=True)
    V, A, rowptr, col = VoronoiMC.apply(X, R, 5)
    rng = np.random.default_rng(0)
    wV = torch.tensor(rng.standard_normal(N), device="cuda")
    wA = torch.tensor(rng.standard_normal(A.shape[0]), device="cuda")
    loss = (V * wV).sum() + (A * wA).sum()
    loss.backward()
    ref = orc.mc_integrate(X.detach().cpu().numpy(), R, 5)
    g0 = orc.mc_adjoint(X.detach().cpu().numpy(), R, 5, ref.hit, ref.l, ref.rowptr, ref.col, wV.cpu().numpy(),
                        wA.cpu().numpy())
    assert np.max(np.abs(X.grad.cpu().numpy() - g0)) <= 1e-10 * np.max(np.abs(g0))


@pytest.mark.parametrize("d,N,R", [(3, 400, 64), (10, 300, 64)])
def test_tensor_wait_limit(orc, d, N, R):
    """The time-out path of the tensor-core kernels' bounded waits, taken on
    purpose: a negative wait limit makes every wait give up before its first
    poll, so the kernel abandons its work, waits (with its own bound) for the
    MMA still in flight, frees its tensor memory and the call reports
    VD_ETIMEOUT.  The device stays usable: a normal call afterwards is
    exact."""
    torch = need_cuda()
    X = synth.uniform(N, d, seed=d)
    cfg = vd.vd_config_default()
    cfg.precision = VD_TC16
    cfg.wait_limit = -1
    ctx = vd.vd_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        vd.vd_set_nodes(ctx, torch.tensor(X, device="cuda"))
        with pytest.raises(vd.VDError) as e:
            vd.vd_mc_free(vd.vd_mc_integrate(ctx, R, 5))
        assert e.value.status == -7  # VD_ETIMEOUT
    finally:
        vd.vd_destroy(ctx)
    torch.cuda.synchronize()
    vor, res, ref = _parity(orc, X, R, seed=5, prec=VD_TC16)
    res.free()
    vor.close()


@pytest.mark.parametrize("d,N,R", [(4, 1500, 64), (16, 400, 32)])
def test_auto_takes_the_fastest_path(orc, d, N, R):
    """VD_AUTO (the default) runs the path measured fastest for the call:
    the tensor-core block walk for node sets without candidate lists
    (d > 8), binary32 screening otherwise.  Same hits, same lengths and the
    same work counters as the explicit choice, and the oracle's hits."""
    need_cuda()
    X = synth.uniform(N, d, seed=60 + d)
    best = VD_TC16 if d > 8 else VD_FP32
    out = []
    for prec in (None, best):
        vor = Voronoi(X) if prec is None else Voronoi(X, precision=prec)
        res = vor.mc_integrate(R, 4)
        out.append((res.hit.cpu().numpy(), res.l.cpu().numpy(), dict(res.stats)))
        res.free()
        vor.close()
    (h0, l0, s0), (h1, l1, s1) = out
    assert np.array_equal(h0, h1) and np.array_equal(l0, l1)
    for k in ("tiles_visited", "pairs_screened", "rechecked", "fallback_rays"):
        assert s0[k] == s1[k], k
    if d > 8:
        assert s0["tiles_visited"] > 0  # the block walk ran
    ref = orc.mc_integrate(X, R, 4)
    assert np.array_equal(h0, ref.hit) and np.array_equal(l0, ref.l)
