"""Pins of the oracle's exact integration from the vertices (Section 3.2,
Algorithms 4-5): volumes and interface areas against scipy's qhull cells
(d = 2, 3), the tiling of the unit cube and the pyramid identity
V_i = (1/d) sum_j h_ij A_ij with A_ij = A_ji (d = 2..5), f = 1 giving V and
A, linear f integrated exactly (the interpolant of a linear function is
itself: V f(centroid), A f(facet centroid), and the cube's integral), the
absolute error bound of Eq. (leibnitz-absolut-error) for sin(x_1^2), and the
MC estimates of Algorithm 3 within a few standard errors of the exact
volumes."""
import numpy as np
import pytest

from brute import face_axis_side
from exact_cells import exact_cells, facet_height
from paper_2405_10050_gb300 import synth


def _fid(a, s):
    return -(2 * a + s + 1)


def _row(rp, col, vals, i):
    return dict(zip(col[rp[i]:rp[i + 1]], vals[rp[i]:rp[i + 1]]))


@pytest.mark.parametrize("d,N", [(2, 80), (3, 50)])
def test_volumes_and_areas_match_qhull(orc, d, N):
    X = synth.uniform(N, d, seed=20 + d)
    T, C, _ = orc.vertices(X)
    V, F, rp, col, A, Fd = orc.leibniz(X, T, C)
    cells = exact_cells(X, _fid)
    for i, c in enumerate(cells):
        assert abs(V[i] - c["volume"]) < 1e-12
        row = _row(rp, col, A, i)
        for j, (a, _) in c["facets"].items():
            assert abs(row[j] - a) < 1e-12
        for j in set(row) - set(c["facets"]):  # facets qhull drops as negligible
            assert row[j] < 1e-12
    assert np.all(np.abs(F - V) < 1e-15)  # f = 1


@pytest.mark.parametrize("d,N", [(2, 100), (3, 60), (4, 40), (5, 25)])
def test_tiling_pyramids_and_symmetry(orc, d, N):
    X = synth.uniform(N, d, seed=30 + d)
    T, C, _ = orc.vertices(X)
    V, F, rp, col, A, Fd = orc.leibniz(X, T, C)
    assert abs(V.sum() - 1.0) < 1e-12
    assert np.all(V > 0)
    for i in range(N):
        s = sum(facet_height(X, i, int(col[q]), face_axis_side) * A[q] for q in range(rp[i], rp[i + 1]))
        assert abs(s / d - V[i]) < 1e-12 * max(1.0, V[i])
        for q in range(rp[i], rp[i + 1]):
            j = int(col[q])
            if j >= 0:
                back = _row(rp, col, A, j)
                assert abs(back[i] - A[q]) <= 1e-11 * max(A[q], 1e-12)
    assert np.all(np.abs(Fd - A) <= 1e-14 * np.maximum(A, 1.0))  # f = 1


@pytest.mark.parametrize("d,N", [(2, 60), (3, 40)])
def test_linear_f_exact(orc, d, N):
    X = synth.uniform(N, d, seed=40 + d)
    T, C, _ = orc.vertices(X)
    b = np.array([1.5, -2.0, 0.75])[:d]
    f = ("poly2", 0.3, list(b), [0.0] * d)
    V, F, rp, col, A, Fd = orc.leibniz(X, T, C, f)
    cells = exact_cells(X, _fid)
    for i, c in enumerate(cells):
        assert abs(F[i] - c["volume"] * (0.3 + b @ c["centroid"])) < 1e-12
        row = _row(rp, col, Fd, i)
        for j, (a, cen) in c["facets"].items():
            assert abs(row[j] - a * (0.3 + b @ cen)) < 1e-12


@pytest.mark.parametrize("d,N", [(4, 40), (5, 20)])
def test_linear_f_over_the_cube(orc, d, N):
    X = synth.uniform(N, d, seed=50 + d)
    T, C, _ = orc.vertices(X)
    b = np.linspace(-1.0, 2.0, d)
    _, F, _, _, _, _ = orc.leibniz(X, T, C, ("poly2", 0.3, list(b), [0.0] * d))
    assert abs(F.sum() - (0.3 + 0.5 * b.sum())) < 1e-12


def test_sin_within_paper_bound_2d(orc):
    from test_oracle_mc_integrals import _exact_2d
    X = synth.uniform(60, 2, seed=61)
    T, C, _ = orc.vertices(X)
    V, F, rp, col, A, Fd = orc.leibniz(X, T, C, ("sin_sq", 0))
    cells = exact_cells(X, _fid)
    for i, c in enumerate(cells):
        exact, _ = _exact_2d(c, X[i], lambda y: np.sin(y[:, 0] ** 2))
        P = np.concatenate(list(c["facet_pts"].values()))
        diam = max(np.linalg.norm(p - q) for p in P for q in P)
        assert abs(F[i] - exact) <= c["volume"] * 6.0 * diam ** 2


@pytest.mark.parametrize("d,N", [(3, 40), (4, 30)])
def test_mc_volumes_against_exact(orc, d, N):
    """Algorithm 3's estimates against the exact volumes of Section 3.2."""
    X = synth.uniform(N, d, seed=70 + d)
    T, C, _ = orc.vertices(X)
    V = orc.leibniz(X, T, C)[0]
    R = 2048
    res = orc.mc_integrate(X, R, seed=5)
    se = orc.sphere_area(d) / d * np.std(res.l ** d, axis=1) / np.sqrt(R)
    z = (res.V - V) / se
    assert np.max(np.abs(z)) < 5.0 and abs(np.mean(z)) < 5.0 / np.sqrt(N)
