"""Pins of the oracle RayCast (Section 2.2, Eq. (t), Algorithm 1)."""
import numpy as np
import pytest

from brute import raycast_numpy
from paper_2405_10050_gb300 import synth

NO_ID = -(2**31)


def test_d1_closed_form(orc):
    """d = 1: from x_i towards +1 the first bisector is the midpoint to the
    next node on the right, else the face x = 1 (and mirrored)."""
    X = np.sort(synth.uniform(50, 1, seed=4), axis=0)
    N = X.shape[0]
    for sign in (+1.0, -1.0):
        dirs = np.full((N, 1), sign)
        hit, t = orc.raycast(X, X, dirs, np.arange(N, dtype=np.int32))
        for i in range(N):
            j = i + 1 if sign > 0 else i - 1
            if 0 <= j < N:
                assert hit[i] == j
                assert abs(t[i] - abs(X[j, 0] - X[i, 0]) / 2) <= 1e-15
            else:
                assert hit[i] == orc.face_id(0, 1 if sign > 0 else 0)
                assert t[i] == ((1.0 if sign > 0 else 0.0) - X[i, 0]) / sign


def test_two_nodes_analytic(orc):
    X = np.array([[0.25, 0.5], [0.75, 0.5]])
    ang = np.linspace(-1.2, 1.2, 25)
    dirs = np.column_stack([np.cos(ang), np.sin(ang)])
    hit, t = orc.raycast(X, np.repeat(X[:1], 25, 0), dirs, np.zeros(25, np.int32))
    # bisector x = 0.5 reached at t = 0.25 / cos(angle) unless a face is closer
    tb = 0.25 / np.cos(ang)
    with np.errstate(divide='ignore'):
        tf = 0.5 / np.abs(dirs[:, 1])  # faces y = 0 / y = 1
    for k in range(25):
        if tb[k] < tf[k]:
            assert hit[k] == 1 and abs(t[k] - tb[k]) < 1e-15
        else:
            assert hit[k] < 0 and abs(t[k] - tf[k]) < 1e-15


@pytest.mark.parametrize("d", [2, 3, 5])
def test_incircle_invariant_and_independent_formula(orc, d):
    """At r* = v + t* u the hit generator and g are equidistant and no node
    is strictly closer (incircle criterion); a numpy evaluation of Eq. (t) in
    another rounding order gives the same hit and t to 1e-12."""
    X = synth.uniform(300, d, seed=d)
    rng = np.random.default_rng(10 + d)
    R = 400
    cells = rng.integers(0, 300, R).astype(np.int32)
    dirs = rng.standard_normal((R, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    hit, t = orc.raycast(X, X[cells], dirs, cells)
    for k in range(R):
        v, u, g = X[cells[k]], dirs[k], X[cells[k]]
        r = v + t[k] * u
        rg = np.linalg.norm(r - g)
        dist = np.linalg.norm(X - r, axis=1)
        assert np.min(dist) >= rg * (1 - 1e-12)
        if hit[k] >= 0:
            assert abs(dist[hit[k]] - rg) <= 1e-12 * max(rg, 1e-300)
        else:
            a = (-hit[k] - 1) >> 1
            assert abs(r[a] - (0.0 if (-hit[k] - 1) & 1 == 0 else 1.0)) < 1e-14
            assert np.all(r > -1e-14) and np.all(r < 1 + 1e-14)
        h2, t2 = raycast_numpy(X, v, u, [int(cells[k])])
        assert h2 == hit[k]
        assert abs(t2 - t[k]) <= 1e-12 * t[k]


def test_eta_excluded_and_vertex_origin(orc):
    """Rays from a vertex along an edge (eta = d generators): the excluded
    generators never come back and the numpy formula agrees."""
    d = 3
    X = synth.uniform(60, d, seed=8)
    tuples, coords, _ = orc.vertices(X)
    rng = np.random.default_rng(3)
    for vid in rng.choice(len(tuples), 60, replace=False):
        sig = tuples[vid]
        for drop in range(d + 1):
            eta = [g for q, g in enumerate(sig) if q != drop]
            if not any(g >= 0 for g in eta):
                continue
            u = orc.search_direction(X, sig, drop)
            nodes = sorted(g for g in eta if g >= 0)
            er = [nodes[0]] + [g for g in eta if g != nodes[0]]
            hit, t = orc.raycast(X, coords[vid][None], u[None], np.array([er], np.int32))
            assert hit[0] not in eta and hit[0] != NO_ID and t[0] > 0
            h2, t2 = raycast_numpy(X, coords[vid], u, er)
            assert h2 == hit[0] and abs(t2 - t[0]) <= 1e-11 * t[0]


def test_box_off_misses(orc):
    X = np.array([[0.5, 0.5]])
    hit, t = orc.raycast(X, X, np.array([[1.0, 0.0]]), np.array([0], np.int32), box=False)
    assert hit[0] == NO_ID and np.isinf(t[0])
    hit, t = orc.raycast(X, X, np.array([[1.0, 0.0]]), np.array([0], np.int32), box=True)
    assert hit[0] == orc.face_id(0, 1) and t[0] == 0.5


def test_tie_break_node_before_face(orc):
    """Equal t: a node (class 0) wins over a face (class 1).  Node 1 sits
    outside the box so that its bisector x = 1 coincides with the face."""
    Xt = np.array([[0.5, 0.5], [1.5, 0.5]])
    hit, t = orc.raycast(Xt, Xt[:1], np.array([[1.0, 0.0]]), np.array([0], np.int32))
    assert t[0] == 0.5 and hit[0] == 1
