"""GPU parity of the RayCast (Section 2.2, Eq. (t), Algorithm 1) against the
FP64 oracle: hit ids bit-exact and t bit-identical (both evaluate Eq. (t) in
binary64 in the same canonical order), for the plain FP64 path, the
binary32-screened path and the tensor-core screened path (rays grouped by
reference node, fp16 MMA over the candidate list), at sizes spanning many
tiles with a ragged tail."""
import numpy as np
import pytest

from gpu_util import clustered_fan, edge_rays, need_cuda, random_unit
from paper_2405_10050_gb300 import NO_ID, VD_FP32, VD_FP64, VD_TC16, Voronoi, synth

pytestmark = pytest.mark.gpu
PRECS = [VD_FP64, VD_FP32, VD_TC16]


def _run(X, O, U, E, prec, box=True, knn_k=0):
    """prec None: the library's default (VD_AUTO)."""
    torch = need_cuda()
    vor = Voronoi(X, box=box, knn_k=knn_k) if prec is None else Voronoi(X, precision=prec, box=box, knn_k=knn_k)
    hit, t, se = vor.raycast(O, U, E, screen_err=True)
    st = vor.stats()
    vor.close()
    return hit.cpu().numpy(), t.cpu().numpy(), se.cpu().numpy(), st


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d,N", [(1, 517), (2, 2049), (3, 3001), (4, 2500), (5, 1999), (7, 1500), (8, 1200),
                                 (12, 800), (16, 1000)])
def test_rays_from_nodes(orc, prec, d, N):
    X = synth.uniform(N, d, seed=100 + d)
    rng = np.random.default_rng(d)
    R = 3000
    cells = rng.integers(0, N, R).astype(np.int32)
    U = random_unit(rng, R, d)
    h0, t0 = orc.raycast(X, X[cells], U, cells)
    h1, t1, se, st = _run(X, X[cells], U, cells[:, None], prec)
    assert np.array_equal(h0, h1)
    assert np.array_equal(t0, t1)
    if prec in (VD_FP32, VD_TC16):
        # (T - t) / t: the binary32 upper bound never undercuts the exact t;
        # its width is set by the absolute binary32 error of the coordinates
        assert np.all(se >= 0) and np.median(se) < 1e-2
        assert st["rechecked"] >= R


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d,N", [(2, 2000), (3, 1500), (5, 3000), (8, 600)])
def test_tree_walk_only(orc, prec, d, N):
    """The bounding-box tree walk alone (no candidate lists) gives the same
    exact hits; with lists a short list forces many rays onto the walk."""
    X = synth.uniform(N, d, seed=200 + d)
    rng = np.random.default_rng(d + 1)
    cells = rng.integers(0, N, 2000).astype(np.int32)
    U = random_unit(rng, 2000, d)
    h0, t0 = orc.raycast(X, X[cells], U, cells)
    for knn in (-1, 4):
        h1, t1, _, st = _run(X, X[cells], U, cells[:, None], prec, knn_k=knn)
        assert np.array_equal(h0, h1) and np.array_equal(t0, t1)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d,N", [(2, 300), (3, 200), (4, 120), (5, 80)])
def test_rays_along_edges(orc, prec, d, N):
    """Rays of the traversal: origin a vertex, eta its d remaining generators."""
    X = synth.uniform(N, d, seed=7 + d)
    tuples, coords, _ = orc.vertices(X)
    O, U, E = edge_rays(orc, X, tuples, coords, 4000, np.random.default_rng(1))
    h0, t0 = orc.raycast(X, O, U, E)
    h1, t1, _, _ = _run(X, O, U, E, prec)
    assert np.array_equal(h0, h1)
    assert np.array_equal(t0, t1)


@pytest.mark.parametrize("prec", PRECS)
def test_gaussian_mixture_nodes(orc, prec):
    X = synth.gaussian_mixture(4000, 6, 8, 0.05, seed=3)
    rng = np.random.default_rng(2)
    cells = rng.integers(0, 4000, 2000).astype(np.int32)
    U = random_unit(rng, 2000, 6)
    h0, t0 = orc.raycast(X, X[cells], U, cells)
    h1, t1, _, _ = _run(X, X[cells], U, cells[:, None], prec)
    assert np.array_equal(h0, h1) and np.array_equal(t0, t1)


@pytest.mark.parametrize("prec", PRECS)
def test_edge_cases(orc, prec):
    # one node: only faces can be hit
    X = np.array([[0.3, 0.6, 0.2]])
    U = random_unit(np.random.default_rng(0), 64, 3)
    h0, t0 = orc.raycast(X, np.repeat(X, 64, 0), U, np.zeros(64, np.int32))
    h1, t1, _, _ = _run(X, np.repeat(X, 64, 0), U, np.zeros((64, 1), np.int32), prec)
    assert np.all(h1 < 0) and np.array_equal(h0, h1) and np.array_equal(t0, t1)
    # exactly one tile, and one tile plus one node
    for N in (32, 33, 64, 1025):
        X = synth.uniform(N, 2, seed=N)
        cells = np.arange(N, dtype=np.int32)
        U = random_unit(np.random.default_rng(N), N, 2)
        h0, t0 = orc.raycast(X, X, U, cells)
        h1, t1, _, _ = _run(X, X, U, cells[:, None], prec)
        assert np.array_equal(h0, h1) and np.array_equal(t0, t1)
    # box off: rays that leave the hull of the nodes miss
    X = synth.uniform(50, 2, seed=5)
    U = random_unit(np.random.default_rng(5), 200, 2)
    cells = np.random.default_rng(6).integers(0, 50, 200).astype(np.int32)
    h0, t0 = orc.raycast(X, X[cells], U, cells, box=False)
    h1, t1, _, _ = _run(X, X[cells], U, cells[:, None], prec, box=False)
    assert np.array_equal(h0, h1) and np.array_equal(t0, t1)
    assert np.any(h1 == NO_ID) and np.all(np.isinf(t1[h1 == NO_ID]))


@pytest.mark.parametrize("prec", [None, VD_FP64, VD_FP32, VD_TC16])
def test_face_behind_a_tiny_direction_component(orc, prec):
    """A node 1e-60 from the face x_1 = 0, rays from it with u_1 = -1e-50:
    u_1 rounds to 0 in binary32, which then bounds nothing, yet the face is
    hit first, at t = 1e-10 (the binary64 recheck has to see it); with
    u_1 = +1e-50 the far face, at t ~ 1e50, must not win.  With candidate
    lists, with the tree walk alone and with a short list."""
    X = synth.uniform(200, 3, seed=11).copy()
    X[0] = [0.5, 1e-60, 0.5]
    th = np.linspace(0.1, 6.0, 8)
    U = np.stack([np.cos(th), np.full(8, -1e-50), np.sin(th)], 1)
    U = np.vstack([U, U * np.array([1.0, -1.0, 1.0])])
    O = np.repeat(X[:1], 16, 0)
    E = np.zeros((16, 1), np.int32)
    h0, t0 = orc.raycast(X, O, U, E)
    assert np.all(h0[:8] == -3) and np.allclose(t0[:8], 1e-10, rtol=1e-15, atol=0)  # face x_1 = 0
    assert np.all(h0[8:] >= 0)
    for knn in (0, -1, 4):
        h1, t1, _, _ = _run(X, O, U, E, prec, knn_k=knn)
        assert np.array_equal(h0, h1) and np.array_equal(t0, t1), f"knn_k={knn}"


def test_host_pointer_path_matches_device(orc):
    """vd_raycast with host (numpy) buffers equals the device-pointer call."""
    need_cuda()
    from paper_2405_10050_gb300 import vd
    X = synth.uniform(700, 3, seed=1)
    rng = np.random.default_rng(3)
    cells = rng.integers(0, 700, 500).astype(np.int32)
    U = random_unit(rng, 500, 3)
    ctx = vd.vd_create(None)
    try:
        vd.vd_set_nodes(ctx, X)
        hit = np.empty(500, np.int32)
        t = np.empty(500)
        vd.vd_raycast(ctx, X[cells], U, cells[:, None].copy(), hit, t)
    finally:
        vd.vd_destroy(ctx)
    h0, t0 = orc.raycast(X, X[cells], U, cells)
    assert np.array_equal(hit, h0) and np.array_equal(t, t0)


def test_invalid_arguments_are_rejected():
    need_cuda()
    from paper_2405_10050_gb300 import VDError, vd
    ctx = vd.vd_create(None)
    try:
        with pytest.raises(VDError):
            vd.vd_set_nodes(ctx, np.zeros((4, 17)))
        with pytest.raises(VDError):
            vd.vd_set_nodes(ctx, np.array([[0.1, np.nan]]))
        Xb = synth.uniform(500, 3, seed=1)
        for v in (np.nan, np.inf):
            Xb[123, 2] = v
            with pytest.raises(VDError):  # one non-finite coordinate among many
                vd.vd_set_nodes(ctx, Xb)
        vd.vd_set_nodes(ctx, synth.uniform(10, 2, seed=0))
        with pytest.raises(VDError):  # eta rows longer than d + 1
            vd.vd_raycast(ctx, np.zeros((1, 2)), np.array([[1.0, 0.0]]), np.zeros((1, 4), np.int32),
                          np.empty(1, np.int32), np.empty(1))
    finally:
        vd.vd_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS)
def test_candidate_overflow_all_rays(orc, prec):
    """Every ray of the fan has more binary32 candidates than its buffer holds
    (far more than R/16 rays): all are redone on the binary64 path and the
    hits equal the oracle's."""
    X, O, U, E = clustered_fan()
    h0, t0 = orc.raycast(X, O, U, E[:, 0])
    assert np.all((h0 >= 1) & (h0 <= 40))  # the cluster is hit
    h1, t1, _, st = _run(X, O, U, E, prec)
    assert np.array_equal(h0, h1) and np.array_equal(t0, t1)
    if prec != VD_FP64:
        assert st["overflow_rays"] > len(O) // 16


def test_tensor_list_wait_limit(orc):
    """The tensor-core list RayCast's time-out path, taken on purpose (a
    negative wait limit gives up before the first poll): the call reports
    VD_ETIMEOUT and every ray it could not finish reads "no hit"; a normal
    call afterwards is exact."""
    torch = need_cuda()
    from paper_2405_10050_gb300 import vd
    X = synth.uniform(2000, 4, seed=41)
    rng = np.random.default_rng(41)
    cells = rng.integers(0, 2000, 3000).astype(np.int32)
    U = random_unit(rng, 3000, 4)
    cfg = vd.vd_config_default()
    cfg.precision = VD_TC16
    cfg.wait_limit = -1
    ctx = vd.vd_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        vd.vd_set_nodes(ctx, torch.tensor(X, device="cuda"))
        hit = torch.zeros(3000, dtype=torch.int32, device="cuda")
        t = torch.zeros(3000, dtype=torch.float64, device="cuda")
        with pytest.raises(vd.VDError) as e:
            vd.vd_raycast(ctx, torch.tensor(X[cells], device="cuda"), torch.tensor(U, device="cuda"),
                          torch.tensor(cells[:, None], device="cuda"), hit, t)
        assert e.value.status == -7  # VD_ETIMEOUT
        assert bool(torch.all(hit == NO_ID))
    finally:
        vd.vd_destroy(ctx)
    torch.cuda.synchronize()
    h0, t0 = orc.raycast(X, X[cells], U, cells)
    h1, t1, _, _ = _run(X, X[cells], U, cells[:, None], VD_TC16)
    assert np.array_equal(h0, h1) and np.array_equal(t0, t1)


@pytest.mark.parametrize("d,N,best", [(2, 1500, VD_FP32), (4, 1500, VD_TC16), (6, 600, VD_TC16)])
def test_auto_takes_the_fastest_path(orc, d, N, best):
    """VD_AUTO (the default) on explicit rays runs the path measured fastest:
    the tensor-core list scan for 3 <= d <= 8, binary32 below.  Same hits and
    the same work counters as the explicit choice, and the oracle's hits."""
    X = synth.uniform(N, d, seed=300 + d)
    rng = np.random.default_rng(d)
    cells = rng.integers(0, N, 3000).astype(np.int32)
    U = random_unit(rng, 3000, d)
    h0, t0 = orc.raycast(X, X[cells], U, cells)
    ha, ta, _, sa = _run(X, X[cells], U, cells[:, None], None)
    hb, tb, _, sb = _run(X, X[cells], U, cells[:, None], best)
    assert np.array_equal(ha, h0) and np.array_equal(ta, t0)
    assert np.array_equal(hb, h0) and np.array_equal(tb, t0)
    for k in ("pairs_screened", "rechecked", "fallback_rays", "launches"):
        assert sa[k] == sb[k], k
