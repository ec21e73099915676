"""Pins of the oracle's random walks on the vertex graph (Section 2.3, the
random walk that approximates the Voronoi graph, with the incircle
RayCast): every step lands on a vertex of the exact set (the pinned
exhaustive traversal, itself checked by brute-force enumeration and qhull),
with its coordinates; consecutive vertices are the two ends of an edge that
holds a node; the edges are taken uniformly among those of the vertex
(chi-square); and enough walkers cover a small diagram completely."""
import numpy as np
import pytest
from scipy import stats

from paper_2405_10050_gb300 import synth


@pytest.mark.parametrize("d,N", [(2, 60), (3, 80), (4, 40), (5, 25)])
def test_walks_stay_on_the_vertex_graph(orc, d, N):
    X = synth.uniform(N, d, seed=80 + d)
    T, C, _ = orc.vertices(X)
    index = {tuple(t): k for k, t in enumerate(T)}
    rng = np.random.default_rng(d)
    start = T[rng.choice(len(T), 24, replace=False)]
    PT, PC = orc.random_walk(X, start, 30, seed=11)
    for w in range(len(start)):
        prev = tuple(start[w])
        for s in range(30):
            cur = tuple(PT[w, s])
            assert cur in index
            assert np.array_equal(PC[w, s], C[index[cur]])
            common = set(prev) & set(cur)
            assert len(common) == d and any(g >= 0 for g in common)
            prev = cur


def test_edges_taken_uniformly(orc):
    X = synth.uniform(300, 3, seed=3)
    T, _, _ = orc.vertices(X)
    start = T[np.random.default_rng(1).choice(len(T), 400, replace=False)]
    PT, _ = orc.random_walk(X, start, 40, seed=5)
    counts = {}
    for w in range(len(start)):
        prev = list(start[w])
        for s in range(40):
            cur = list(PT[w, s])
            valid = [q for q in range(4) if any(g >= 0 for k, g in enumerate(prev) if k != q)]
            dropped = [q for q in range(4) if prev[q] not in cur]
            assert len(dropped) == 1 and dropped[0] in valid
            counts.setdefault(len(valid), np.zeros(4, np.int64))[valid.index(dropped[0])] += 1
            prev = cur
    full = counts[4]
    assert stats.chisquare(full).pvalue > 1e-3


def test_walkers_cover_a_small_diagram(orc):
    X = synth.uniform(30, 2, seed=7)
    T, _, _ = orc.vertices(X)
    start = np.repeat(T[:1], 64, axis=0)
    PT, _ = orc.random_walk(X, start, 200, seed=3)
    seen = set(map(tuple, PT.reshape(-1, 3)))
    assert seen == set(map(tuple, T))
