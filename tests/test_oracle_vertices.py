"""Pins of the oracle's exhaustive traversal (Algorithm 2, Section 2.3) with
the box faces as generators."""
import json
import os
from collections import Counter

import numpy as np
import pytest
from scipy.spatial import Delaunay

from brute import face_axis_side, vertices_bruteforce
from paper_2405_10050_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _edges(tuples, d):
    """edge (d-subset with >= 1 node) -> number of vertices containing it"""
    cnt = Counter()
    for sig in map(tuple, tuples):
        for q in range(d + 1):
            eta = sig[:q] + sig[q + 1:]
            if any(g >= 0 for g in eta):
                cnt[eta] += 1
    return cnt


@pytest.mark.parametrize("d,N,seed", [(2, 6, 0), (2, 12, 1), (2, 12, 2), (3, 7, 3), (3, 10, 4), (4, 7, 5)])
def test_traversal_equals_bruteforce_enumeration(orc, d, N, seed):
    X = synth.uniform(N, d, seed=seed)
    tuples, coords, stats = orc.vertices(X)
    brute = vertices_bruteforce(X)
    assert sorted(map(tuple, tuples)) == brute
    assert stats["rediscoveries"] == 0 and stats["ties"] == 0


@pytest.mark.parametrize("d,N", [(2, 200), (3, 150), (4, 60)])
def test_vertex_invariants(orc, d, N):
    X = synth.uniform(N, d, seed=17 + d)
    tuples, coords, stats = orc.vertices(X)
    V = len(tuples)
    # every vertex: equidistant to its nodes, none closer, on its faces, in the box
    for sig, r in zip(tuples, coords):
        nodes = [g for g in sig if g >= 0]
        dist = np.linalg.norm(X - r, axis=1)
        R = dist[nodes[0]]
        assert np.all(np.abs(dist[nodes] - R) <= 1e-12 * max(R, 1e-3))
        assert np.min(dist) >= R * (1 - 1e-12)
        for g in sig:
            if g < 0:
                a, s = face_axis_side(g)
                assert r[a] == float(s)
        assert np.all(r >= -1e-13) and np.all(r <= 1 + 1e-13)
    # every edge has exactly two endpoints (Section 2.3)
    cnt = _edges(tuples, d)
    assert set(cnt.values()) == {2}
    # each of the 2^d box corners appears once
    corners = [sig for sig in tuples if sum(g < 0 for g in sig) == d]
    assert len(corners) == 2 ** d
    assert len({tuple(coords[i]) for i in range(V) if sum(g < 0 for g in tuples[i]) == d}) == 2 ** d
    # Alg. 2 with the edge counter casts one ray per vertex except the seed
    assert stats["raycasts"] == V - 1


def test_euler_characteristic_d2(orc):
    """Planar clipped diagram: V - E + (N + 1) = 2."""
    for seed in range(3):
        X = synth.uniform(300, 2, seed=seed)
        tuples, _, _ = orc.vertices(X)
        E = len(_edges(tuples, 2))
        assert len(tuples) - E + 300 == 1


def test_node_tuples_match_qhull_delaunay(orc):
    """Vertices with only node generators are exactly the Delaunay simplices
    (scipy / qhull) whose circumcentre lies inside the box."""
    d, N = 3, 2000
    X = synth.uniform(N, d, seed=0)
    tuples, coords, _ = orc.vertices(X)
    mine = {tuple(s) for s in tuples if min(s) >= 0}
    tri = Delaunay(X)
    ref, borderline = set(), 0
    for simp in tri.simplices:
        P = X[simp]
        A = 2.0 * (P[1:] - P[0])
        b = np.sum(P[1:] ** 2, axis=1) - np.sum(P[0] ** 2)
        c = np.linalg.solve(A, b)
        m = min(c.min(), 1 - c.max())
        if abs(m) < 1e-9:
            borderline += 1
            continue
        if m > 0:
            ref.add(tuple(sorted(simp)))
    assert borderline == 0
    assert mine == ref


def test_paper_table_sanity(orc):
    """Loose check against the paper's table of vertices and neighbours per
    cell (the table's own numbers are approximate and periodic)."""
    with open(os.path.join(GOLDEN, "paper_tables.json")) as f:
        tab = json.load(f)["vertices_neighbors_per_cell"]
    for d, N in [(2, 3000), (3, 2000)]:
        X = synth.uniform(N, d, seed=1)
        tuples, _, _ = orc.vertices(X)
        interior = np.all((X > 0.2) & (X < 0.8), axis=1)
        vcount, nbrs = Counter(), {i: set() for i in range(N)}
        for sig in tuples:
            nodes = [g for g in sig if g >= 0]
            for g in nodes:
                vcount[g] += 1
                nbrs[g].update(h for h in nodes if h != g)
        idx = np.nonzero(interior)[0]
        mv = np.mean([vcount[i] for i in idx])
        mn = np.mean([len(nbrs[i]) for i in idx])
        assert abs(mv / tab["vertices"][str(d)] - 1) < 0.25
        assert abs(mn / tab["neighbors"][str(d)] - 1) < 0.25


def test_search_direction_and_coords(orc):
    d = 4
    X = synth.uniform(40, d, seed=9)
    tuples, coords, _ = orc.vertices(X)
    for sig, r in zip(tuples[:50], coords[:50]):
        r2 = orc.vertex_coords(X, sig)
        assert np.array_equal(r2, r)
        for drop in range(d + 1):
            eta = [g for q, g in enumerate(sig) if q != drop]
            if not any(g >= 0 for g in eta):
                assert orc.search_direction(X, sig, drop) is None
                continue
            u = orc.search_direction(X, sig, drop)
            assert abs(np.linalg.norm(u) - 1) < 1e-14
            nodes = [g for g in eta if g >= 0]
            for k in nodes[1:]:
                assert abs(u @ (X[k] - X[nodes[0]])) < 1e-12
            for g in eta:
                if g < 0:
                    assert u[face_axis_side(g)[0]] == 0.0
            e = sig[drop]
            if e >= 0:
                assert u @ (X[e] - X[nodes[0]]) < 0
            else:
                a, s = face_axis_side(e)
                assert (u[a] > 0) if s == 0 else (u[a] < 0)
