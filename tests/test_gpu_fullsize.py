"""Parity at the full workload sizes, in the launch configuration the
benchmark times, on outputs the oracle computes one by one:

* exhaustive traversal (Algorithm 2), N = 20000 uniform nodes in [0,1]^5:
  the screened and the binary64 paths give the same tuples and coordinates;
  sampled vertices are re-solved by the oracle and every edge of them is
  re-cast by the oracle's brute-force RayCast, whose far end must be a vertex
  of the set; every edge of the whole set has exactly two endpoints and each
  cube corner appears once;
* Monte Carlo (Algorithm 3), N = 100000 uniform nodes in [0,1]^4, 1024 rays
  per cell (with the function integrals F_V, F_d of sin(x_1^2), 2 samples
  per ray, on sampled cells), and N = 200000 nodes in [0,1]^16 from a 32-component Gaussian
  mixture (sigma 0.1), 64 rays per cell: sampled rays equal the oracle's
  brute-force RayCast (hit id and l bit for bit), and the binary32, tensor
  core and binary64 paths agree on every ray;
* batched Monte Carlo, 512 sets of uneven N and d: sampled rays of sampled
  sets equal the oracle with the set's own Philox set id.
"""
import numpy as np
import pytest

from gpu_util import need_cuda
from paper_2405_10050_gb300 import VD_FP32, VD_FP64, VD_TC16, Voronoi, synth, vd

pytestmark = pytest.mark.gpu


def _find_row(T, row):
    """Binary search of a row in lexicographically sorted int32 rows."""
    lo, hi = 0, len(T)
    key = tuple(int(v) for v in row)
    while lo < hi:
        mid = (lo + hi) // 2
        if tuple(int(v) for v in T[mid]) < key:
            lo = mid + 1
        else:
            hi = mid
    return lo < len(T) and tuple(int(v) for v in T[lo]) == key


def _edge_endpoint_counts_are_two(T, d):
    """Each edge (a vertex tuple minus one entry, holding at least one node)
    belongs to exactly two vertices."""
    keys = []
    for q in range(d + 1):
        E = np.delete(T, q, axis=1).astype(np.int64) + 16  # ids >= -2d-1 > -16
        E = E[np.any(E >= 16, axis=1)]
        keys.append(E)
    E = np.concatenate(keys)
    k1 = np.zeros(len(E), np.uint64)
    for c in range(min(d, 4)):
        k1 = (k1 << np.uint64(15)) | E[:, c].astype(np.uint64)
    k2 = np.zeros(len(E), np.uint64)
    for c in range(4, d):
        k2 = (k2 << np.uint64(15)) | E[:, c].astype(np.uint64)
    o = np.lexsort((k2, k1))
    k1, k2 = k1[o], k2[o]
    if len(k1) % 2:
        return False
    pair_eq = (k1[0::2] == k1[1::2]) & (k2[0::2] == k2[1::2])
    nxt_ne = (k1[1:-1:2] != k1[2::2]) | (k2[1:-1:2] != k2[2::2])
    return bool(np.all(pair_eq) and np.all(nxt_ne))


def test_traversal_d5_n20000(orc):
    need_cuda()
    d, N = 5, 20000
    assert N < 2 ** 15
    X = synth.uniform(N, d, seed=0)
    out = {}
    for prec in (VD_FP32, VD_FP64, VD_TC16):
        vor = Voronoi(X, precision=prec)
        t, c, st = vor.vertices()
        out[prec] = (t.cpu().numpy(), c.cpu().numpy(), st)
        vor.close()
    T, C, st = out[VD_FP32]
    for other in (VD_FP64, VD_TC16):
        assert np.array_equal(T, out[other][0]) and np.array_equal(C, out[other][1])
    # the per-cell exploration (cells in index order, 1024 at a time, the edge
    # table rebuilt per batch) finds the same vertices with a smaller edge table
    vor = Voronoi(X)
    t, c, stc = vor.vertices(cells_per_batch=1024)
    vor.close()
    assert np.array_equal(T, t.cpu().numpy()) and np.array_equal(C, c.cpu().numpy())
    assert stc["edge_table_bytes"] * 4 < st["edge_table_bytes"]
    assert st["vertices"] == len(T) > 2_000_000
    assert np.all(np.diff(T, axis=1) > 0)  # each tuple sorted, no repeats
    assert int(np.sum(np.sum(T < 0, axis=1) == d)) == 2 ** d  # the cube corners
    assert _edge_endpoint_counts_are_two(T, d)
    rng = np.random.default_rng(1)
    for vid in rng.choice(len(T), 60, replace=False):
        sig = T[vid]
        r = orc.vertex_coords(X, sig)
        assert r is not None and np.array_equal(r, C[vid])
        for drop in range(d + 1):
            eta = [int(g) for q, g in enumerate(sig) if q != drop]
            nodes = sorted(g for g in eta if g >= 0)
            if not nodes:
                continue
            u = orc.search_direction(X, sig, drop)
            e = np.array([[nodes[0]] + [g for g in eta if g != nodes[0]]], np.int32)
            hit, _ = orc.raycast(X, C[vid][None, :], u[None, :], e)
            nb = np.array(sorted(eta + [int(hit[0])]), np.int32)
            assert _find_row(T, nb), (sig, drop, nb)


def _mc_sample_check(orc, X, R, seed, hit, l, cells, rays_per_cell, rng, set_id=0):
    """hit, l: host arrays of the sampled cells' rows [len(cells), R]."""
    d = X.shape[1]
    for row, i in enumerate(cells):
        U = orc.mc_directions(seed, set_id, 1, R, d, cell0=int(i))[0]
        ks = np.arange(R) if rays_per_cell >= R else np.sort(rng.choice(R, rays_per_cell, replace=False))
        O = np.repeat(X[i][None, :], len(ks), axis=0)
        E = np.full((len(ks), 1), int(i), np.int32)
        h0, t0 = orc.raycast(X, O, U[ks], E)
        assert np.array_equal(hit[row, ks], h0), (i, set_id)
        assert np.array_equal(l[row, ks], t0), (i, set_id)


def _integrals_sample_check(orc, X, R, seed, res, cells, idx, m=2):
    """Algorithm 3's F_V and F_d of f = sin(x_1^2) (m samples per ray) of the
    whole set, compared on the sampled cells with the oracle's sums over the
    same rays (within 1e-12 relative: every term is positive)."""
    FV, Fd = res.integrals(vd.func_sin_sq(0), m)
    rp = res.rowptr.cpu().numpy()
    col = res.col.cpu().numpy()
    Fd = Fd.cpu().numpy()
    lrp = np.concatenate([[0], np.cumsum([rp[i + 1] - rp[i] for i in cells])])
    lcol = np.concatenate([col[rp[i]:rp[i + 1]] for i in cells])
    FV0, Fd0 = orc.mc_integrals(X, R, seed, cells, res.hit[idx].cpu().numpy(), res.l[idx].cpu().numpy(), lrp, lcol,
                                ("sin_sq", 0), m)
    FVs = FV[idx].cpu().numpy()
    Fds = np.concatenate([Fd[rp[i]:rp[i + 1]] for i in cells])
    assert np.all(np.abs(FVs - FV0) <= 1e-12 * np.abs(FV0) + 1e-300)
    assert np.all(np.abs(Fds - Fd0) <= 1e-12 * np.abs(Fd0) + 1e-300)


def _mc_full(X, R, seed, prec):
    vor = Voronoi(X, precision=prec)
    return vor, vor.mc_integrate(R, seed)


def test_mc_d4_n100000(orc):
    torch = need_cuda()
    N, d, R, seed = 100000, 4, 1024, 7
    X = synth.uniform(N, d, seed=0)
    rng = np.random.default_rng(2)
    cells = np.concatenate([[0, N - 1], rng.choice(N, 10, replace=False)])
    base = None
    for prec in (VD_FP32, VD_TC16, VD_FP64):
        vor, res = _mc_full(X, R, seed, prec)
        if base is None:
            base, vbase = res, vor
            assert abs(float(res.V.sum()) - 1.0) < 5e-3  # sum of volumes of the unit cube
            idx = torch.tensor(cells, device="cuda")
            h = res.hit[idx].cpu().numpy()
            l = res.l[idx].cpu().numpy()
            _mc_sample_check(orc, X, R, seed, h[:2], l[:2], cells[:2], R, rng)
            _mc_sample_check(orc, X, R, seed, h[2:], l[2:], cells[2:], 48, rng)
            _integrals_sample_check(orc, X, R, seed, res, cells, idx)
        else:
            assert torch.equal(res.hit, base.hit) and torch.equal(res.l, base.l)
            assert torch.equal(res.rowptr, base.rowptr) and torch.equal(res.col, base.col)
            res.free()
            vor.close()
    base.free()
    vbase.close()


def test_mc_d16_n200000_mixture(orc):
    torch = need_cuda()
    N, d, R, seed = 200000, 16, 64, 5
    X = synth.gaussian_mixture(N, d, K=32, sigma=0.1, seed=0)
    rng = np.random.default_rng(3)
    cells = rng.choice(N, 6, replace=False)
    base = None
    for prec in (VD_TC16, VD_FP32):
        vor, res = _mc_full(X, R, seed, prec)
        if base is None:
            base, vbase = res, vor
            idx = torch.tensor(cells, device="cuda")
            _mc_sample_check(orc, X, R, seed, res.hit[idx].cpu().numpy(), res.l[idx].cpu().numpy(), cells, 12,
                             rng)
        else:
            assert torch.equal(res.hit, base.hit) and torch.equal(res.l, base.l)
            res.free()
            vor.close()
    base.free()
    vbase.close()


def test_batch_512_sets(orc):
    torch = need_cuda()
    sets = synth.batch_sets(512, seed=0)
    R, seed = 256, 3
    ctx = vd.vd_create(None, torch.cuda.current_stream().cuda_stream)
    try:
        Xd = [torch.tensor(X, device="cuda") for X, _ in sets]
        mcs = vd.vd_mc_integrate_batch(ctx, Xd, R, seed)
        rng = np.random.default_rng(4)
        for s in [0, 255, 256, 511] + list(rng.choice(512, 4, replace=False)):
            X = sets[s][0]
            N = X.shape[0]
            hit = np.empty((N, R), np.int32)
            l = np.empty((N, R))
            vd.vd_mc_rays(mcs[s], hit, l)
            cells = rng.choice(N, min(N, 5), replace=False)
            _mc_sample_check(orc, X, R, seed, hit[cells], l[cells], cells, 16, rng, set_id=int(s))
        for mc in mcs:
            vd.vd_mc_free(mc)
    finally:
        vd.vd_destroy(ctx)
