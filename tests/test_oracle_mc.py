"""Pins of the oracle's Monte Carlo volumes, areas (Section 3.1, Algorithm 3)
and of their adjoint."""
import json
import os

import numpy as np
import pytest

from brute import face_axis_side
from exact_cells import exact_cells, exact_volume_gradient, facet_height
from paper_2405_10050_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_sphere_area_closed_forms(orc):
    with open(os.path.join(GOLDEN, "paper_tables.json")) as f:
        vals = json.load(f)["sphere_area"]["values"]
    for d, v in vals.items():
        assert abs(orc.sphere_area(int(d)) - v) <= 1e-15 * v


def test_d1_closed_form(orc):
    """d = 1, S_0 = 2: V_i = (2/R)(n_+ l_+ + n_- l_-), A to each side =
    (2/R) n_pm, with l_pm the distance to the bisector or face on that side."""
    X = np.sort(synth.uniform(20, 1, seed=2), axis=0)
    R = 64
    res = orc.mc_integrate(X, R, seed=5)
    u = orc.mc_directions(5, 0, 20, R, 1)[:, :, 0]
    for i in range(20):
        lp = (X[i + 1, 0] - X[i, 0]) / 2 if i + 1 < 20 else 1 - X[i, 0]
        lm = (X[i, 0] - X[i - 1, 0]) / 2 if i > 0 else X[i, 0]
        npos = int(np.sum(u[i] > 0))
        assert abs(res.V[i] - (2.0 / R) * (npos * lp + (R - npos) * lm)) < 1e-15
        row = dict(zip(res.col[res.rowptr[i]:res.rowptr[i + 1]], res.A[res.rowptr[i]:res.rowptr[i + 1]]))
        right = i + 1 if i + 1 < 20 else -2
        if npos:
            assert abs(row[right] - 2.0 * npos / R) < 1e-15


@pytest.mark.parametrize("d", [2, 3, 5])
def test_pyramid_identity_per_estimate(orc, d):
    """V_i = (1/d) sum_j h_ij A_ij holds for the estimates themselves
    (Section 3.3 uses it for HMC volumes): h_ij is |x_j - x_i|/2 for a node
    and the distance to the face for a box face."""
    X = synth.uniform(80, d, seed=d)
    res = orc.mc_integrate(X, 64, seed=1)
    for i in range(80):
        s = 0.0
        for q in range(res.rowptr[i], res.rowptr[i + 1]):
            s += facet_height(X, i, int(res.col[q]), face_axis_side) * res.A[q]
        assert abs(s / d - res.V[i]) <= 1e-12 * res.V[i]


@pytest.mark.parametrize("d,N", [(2, 60), (3, 40)])
def test_mc_converges_to_exact_polytopes(orc, d, N):
    """Exact cells from qhull; the estimate of every volume is within a few
    standard errors (SE from the per-ray l^d spread), volumes sum to ~1 and
    the exact cells tile the box."""
    X = synth.uniform(N, d, seed=21 + d)
    cells = exact_cells(X, lambda a, s: -(2 * a + s + 1))
    Vex = np.array([c["volume"] for c in cells])
    assert abs(Vex.sum() - 1.0) < 1e-12
    for i, c in enumerate(cells):  # pyramid identity on the exact cells
        s = sum(facet_height(X, i, j, face_axis_side) * A for j, (A, _) in c["facets"].items())
        assert abs(s / d - c["volume"]) < 1e-11
    R = 4096
    res = orc.mc_integrate(X, R, seed=3)
    ld = res.l ** d
    S = orc.sphere_area(d)
    se = S / d * np.std(ld, axis=1) / np.sqrt(R)
    z = (res.V - Vex) / se
    assert np.max(np.abs(z)) < 5.0
    assert abs(np.mean(z)) < 5.0 / np.sqrt(N)
    assert abs(res.V.sum() - 1.0) < 5 * np.sqrt(np.sum(se ** 2))
    # areas: every exact facet with a sizeable area is found, and the
    # estimates are unbiased in aggregate
    zs = []
    for i, c in enumerate(cells):
        row = dict(zip(res.col[res.rowptr[i]:res.rowptr[i + 1]], res.A[res.rowptr[i]:res.rowptr[i + 1]]))
        assert set(row) <= set(c["facets"])
        tot = sum(A for A, _ in c["facets"].values())
        for j, (A, _) in c["facets"].items():
            if A > 0.05 * tot:
                assert j in row
                zs.append((row[j] - A) / A)
    assert abs(np.mean(zs)) < 0.02


def test_adjoint_matches_finite_differences(orc):
    """Adjoint of the estimator with directions and argmins fixed against
    central differences of the same estimator (rel 1e-4)."""
    for d in (2, 3, 4):
        N, R = 25, 32
        X = synth.uniform(N, d, seed=40 + d)
        res = orc.mc_integrate(X, R, seed=7)
        rng = np.random.default_rng(d)
        gV = rng.standard_normal(N)
        gA = rng.standard_normal(res.col.shape[0])
        gX = orc.mc_adjoint(X, R, 7, res.hit, res.l, res.rowptr, res.col, gV, gA)
        h = 1e-6
        fd = np.zeros_like(X)
        for k in range(N):
            for a in range(d):
                Xp, Xm = X.copy(), X.copy()
                Xp[k, a] += h
                Xm[k, a] -= h
                Vp, Ap = orc.mc_eval_fixed(Xp, R, 7, res.hit, res.rowptr, res.col)
                Vm, Am = orc.mc_eval_fixed(Xm, R, 7, res.hit, res.rowptr, res.col)
                fd[k, a] = (gV @ (Vp - Vm) + gA @ (Ap - Am)) / (2 * h)
        assert np.max(np.abs(gX - fd)) <= 1e-4 * np.max(np.abs(fd))
        # the fixed-argmin estimator reproduces the forward pass exactly
        V0, A0 = orc.mc_eval_fixed(X, R, 7, res.hit, res.rowptr, res.col)
        assert np.allclose(V0, res.V, rtol=1e-14, atol=0) and np.allclose(A0, res.A, rtol=1e-13, atol=0)


@pytest.mark.parametrize("d,N", [(2, 30), (3, 30)])
def test_volume_gradient_is_unbiased(orc, d, N):
    """dV/dX from the MC adjoint (16 independent seeds, batch means) against
    the exact polytope gradient; also sum_i dV_i/dx_k = 0 for the exact one."""
    X = synth.uniform(N, d, seed=60 + d)
    cells = exact_cells(X, lambda a, s: -(2 * a + s + 1))
    G = exact_volume_gradient(X, cells)
    assert np.max(np.abs(G.sum(axis=0))) < 1e-12
    gV = np.random.default_rng(1).standard_normal(N)
    exact = np.einsum("i,ikd->kd", gV, G)
    ests = []
    for seed in range(16):
        res = orc.mc_integrate(X, 1024, seed=100 + seed)
        ests.append(orc.mc_adjoint(X, 1024, 100 + seed, res.hit, res.l, res.rowptr, res.col, gV,
                                   np.zeros(res.col.shape[0])))
    ests = np.array(ests)
    mean = ests.mean(axis=0)
    se = ests.std(axis=0, ddof=1) / 4.0
    z = (mean - exact) / se
    assert np.max(np.abs(z)) < 5.5
    assert abs(z.mean()) < 5.0 / np.sqrt(z.size)
