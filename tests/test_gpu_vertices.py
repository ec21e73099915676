"""GPU parity of the exhaustive vertex traversal (Section 2.3, Algorithm 2)
against the oracle's sequential traversal: the sorted tuple sets are
identical and the coordinates, solved from the tuples in binary64 in the
same order on both sides, are bit-identical."""
from collections import Counter

import numpy as np
import pytest

from gpu_util import need_cuda
from paper_2405_10050_gb300 import VD_FP32, VD_FP64, VD_TC16, Voronoi, synth

pytestmark = pytest.mark.gpu


def _gpu_vertices(X, prec):
    need_cuda()
    vor = Voronoi(X, precision=prec)
    t, c, st = vor.vertices()
    vor.close()
    return t.cpu().numpy(), c.cpu().numpy(), st


@pytest.mark.parametrize("prec", [VD_FP64, VD_FP32, VD_TC16])
@pytest.mark.parametrize("d,N", [(2, 500), (3, 2000), (4, 300), (5, 120), (6, 40)])
def test_vertices_parity(orc, prec, d, N):
    X = synth.uniform(N, d, seed=0)
    t0, c0, _ = orc.vertices(X)
    t1, c1, st = _gpu_vertices(X, prec)
    assert t1.shape == t0.shape
    assert np.array_equal(t1, t0)
    assert np.array_equal(c1, c0)
    assert st["vertices"] == len(t0) and st["levels"] >= 1


@pytest.mark.parametrize("prec", [VD_FP64, VD_FP32, VD_TC16])
def test_vertices_mixture_and_tiny(orc, prec):
    for X in [synth.gaussian_mixture(400, 3, 8, 0.05, seed=2), synth.uniform(1, 2, seed=1),
              synth.uniform(2, 3, seed=2), synth.uniform(33, 2, seed=3)]:
        t0, c0, _ = orc.vertices(X)
        t1, c1, _ = _gpu_vertices(X, prec)
        assert np.array_equal(t1, t0) and np.array_equal(c1, c0)


@pytest.mark.parametrize("prec", [VD_FP64, VD_FP32, VD_TC16])
@pytest.mark.parametrize("d,N,batch", [(2, 500, 1), (2, 500, 37), (3, 2000, 100), (4, 300, 7), (5, 120, 16),
                                       (6, 40, 1), (6, 40, 0)])
def test_cell_exploration_parity(orc, prec, d, N, batch):
    """Per-cell sequential exploration (Section 2.3): cells in index order,
    `batch` at a time (1: one cell at a time, 0: automatic), the edge counters
    rebuilt for each batch from the vertices found so far: the same tuples
    and coordinates as the oracle's traversal, bit for bit, with a smaller
    edge table than the whole-diagram traversal's."""
    need_cuda()
    X = synth.uniform(N, d, seed=0)
    t0, c0, _ = orc.vertices(X)
    vor = Voronoi(X, precision=prec)
    t1, c1, st = vor.vertices(cells_per_batch=batch)
    _, _, st_all = vor.vertices()
    vor.close()
    assert np.array_equal(t1.cpu().numpy(), t0) and np.array_equal(c1.cpu().numpy(), c0)
    assert st["vertices"] == len(t0)
    assert 0 < st["edge_table_bytes"] < st_all["edge_table_bytes"]
    assert st["vertex_table_bytes"] == st_all["vertex_table_bytes"]


@pytest.mark.parametrize("prec", [VD_FP32, VD_TC16])
def test_cell_exploration_mixture_and_tiny(orc, prec):
    """Clustered nodes (cells of very different sizes; most batch cells are
    reached from their neighbours' vertices, not seeded), one and two nodes,
    33 nodes in batches of 5 (a ragged last batch)."""
    need_cuda()
    for X, b in [(synth.gaussian_mixture(400, 3, 8, 0.05, seed=2), 50), (synth.uniform(1, 2, seed=1), 1),
                 (synth.uniform(2, 3, seed=2), 1), (synth.uniform(33, 2, seed=3), 5)]:
        t0, c0, _ = orc.vertices(X)
        vor = Voronoi(X, precision=prec)
        t1, c1, _ = vor.vertices(cells_per_batch=b)
        vor.close()
        assert np.array_equal(t1.cpu().numpy(), t0) and np.array_equal(c1.cpu().numpy(), c0)


def test_vertex_invariants_larger(orc):
    """d = 5, N = 3000: every edge has two endpoints and each of the 2^d
    corners appears once; a sample of vertices is checked by the oracle's
    brute force (equidistant, no node closer)."""
    d, N = 5, 3000
    X = synth.uniform(N, d, seed=4)
    t, c, st = _gpu_vertices(X, VD_FP32)
    cnt = Counter()
    for sig in map(tuple, t):
        for q in range(d + 1):
            eta = sig[:q] + sig[q + 1:]
            if any(g >= 0 for g in eta):
                cnt[eta] += 1
    assert set(cnt.values()) == {2}
    assert sum(1 for sig in t if np.sum(sig < 0) == d) == 2 ** d
    rng = np.random.default_rng(0)
    for v in rng.choice(len(t), 300, replace=False):
        r = orc.vertex_coords(X, t[v])
        assert np.array_equal(r, c[v])
        nodes = [g for g in t[v] if g >= 0]
        dist = np.linalg.norm(X - r, axis=1)
        R = dist[nodes[0]]
        assert np.min(dist) >= R * (1 - 1e-12)


def test_context_reuse_across_sizes(orc):
    """One context, node sets of growing and shrinking size and dimension:
    the traversal and MC work buffers kept in the context are reused or
    grown, and every result still equals the oracle's."""
    need_cuda()
    vor = Voronoi(synth.uniform(900, 3, seed=1), precision=VD_FP32)
    try:
        for X in [synth.uniform(900, 3, seed=1), synth.uniform(40, 2, seed=2), synth.uniform(2500, 3, seed=3),
                  synth.gaussian_mixture(150, 4, 4, 0.1, seed=4), synth.uniform(900, 3, seed=1)]:
            vor.set_nodes(X)
            t1, c1, _ = vor.vertices()
            t0, c0, _ = orc.vertices(X)
            assert np.array_equal(t1.cpu().numpy(), t0) and np.array_equal(c1.cpu().numpy(), c0)
            R = 48 if X.shape[0] < 1000 else 16
            res = vor.mc_integrate(R, 9)
            ref = orc.mc_integrate(X, R, 9)
            assert np.array_equal(res.hit.cpu().numpy(), ref.hit)
            assert np.array_equal(res.l.cpu().numpy(), ref.l)
            res.free()
    finally:
        vor.close()
