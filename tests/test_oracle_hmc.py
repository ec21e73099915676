"""Pins of the oracle's heuristic Monte Carlo integration (Section 3.3):
volumes from the interface areas, interface integrals from the interface's
vertices and their mean, cell integrals by the cone rule of Eq.
(leibniz-int).

* f = 1 turns every formula into the MC estimates themselves: F = A exactly,
  V_H = (1/d) sum_j h_ij A_ij = the MC volume (the per-estimate pyramid
  identity), I_H = V_H; every interface has at least d vertices.
* d = 2 with exact inputs (qhull facet lengths, the oracle's pinned vertex
  set): an interface is a segment [a, b] with mean m, so for linear f both
  the interface rule and the cone rule are exact (F = |e| f(m), I = the exact
  integral V f(centroid)); for a quadratic f the interface rule is
  |e| (f(a) + f(b) + f(m)) / 3 while Simpson's rule is exact, which differ by
  |e| Q(e) / 12 (Q the quadratic part, e = b - a).
* f = sin(x_1^2): the cell integrals stay within the absolute bound
  |C| sup|f''| diam(C)^2 of Eq. (leibnitz-absolut-error) of the exact
  integrals (Gauss-Legendre over the fan triangles)."""
import numpy as np
import pytest

from exact_cells import exact_cells, facet_height
from brute import face_axis_side
from paper_2405_10050_gb300 import synth


def _fid(a, s):
    return -(2 * a + s + 1)


def _exact_csr(cells):
    rowptr, col, A = [0], [], []
    for c in cells:
        for j in sorted(c["facets"]):
            col.append(j)
            A.append(c["facets"][j][0])
        rowptr.append(len(col))
    return np.array(rowptr, np.int64), np.array(col, np.int32), np.array(A)


@pytest.mark.parametrize("d", [2, 3, 5])
def test_f_one_gives_the_mc_estimates(orc, d):
    X = synth.uniform(60 if d < 5 else 25, d, seed=50 + d)
    res = orc.mc_integrate(X, 256, seed=6)
    T, C, _ = orc.vertices(X)
    VH, FH, IH, K = orc.hmc(X, res.rowptr, res.col, res.A, T, C, ("one",))
    assert np.array_equal(FH, res.A)
    assert np.all(np.abs(VH - res.V) <= 1e-12 * res.V)
    assert np.all(np.abs(IH - VH) <= 1e-12 * VH)
    assert np.all(K >= d)


def test_linear_f_exact_in_2d(orc):
    X = synth.uniform(50, 2, seed=71)
    cells = exact_cells(X, _fid)
    rowptr, col, A = _exact_csr(cells)
    T, C, _ = orc.vertices(X)
    f = ("poly2", 0.4, [2.0, -1.5], [0.0, 0.0])
    b = np.array([2.0, -1.5])
    VH, FH, IH, K = orc.hmc(X, rowptr, col, A, T, C, f)
    assert np.all(K == 2)
    for i, c in enumerate(cells):
        assert abs(IH[i] - c["volume"] * (0.4 + b @ c["centroid"])) < 1e-12
        assert abs(VH[i] - c["volume"]) < 1e-12
        for q in range(rowptr[i], rowptr[i + 1]):
            Ae, cen = c["facets"][int(col[q])]
            assert abs(FH[q] - Ae * (0.4 + b @ cen)) < 1e-12


def test_quadratic_interfaces_2d(orc):
    X = synth.uniform(50, 2, seed=72)
    cells = exact_cells(X, _fid)
    rowptr, col, A = _exact_csr(cells)
    T, C, _ = orc.vertices(X)
    c0, bv, qv = 0.1, np.array([0.5, 1.0]), np.array([3.0, -2.0])
    f = ("poly2", c0, list(bv), list(qv))
    g = lambda y: c0 + y @ bv + (y * y) @ qv
    _, FH, _, _ = orc.hmc(X, rowptr, col, A, T, C, f)
    for i, c in enumerate(cells):
        for q in range(rowptr[i], rowptr[i + 1]):
            a, bb = c["facet_pts"][int(col[q])]
            e = bb - a
            L = np.linalg.norm(e)
            simpson = L * (g(a) + 4 * g(0.5 * (a + bb)) + g(bb)) / 6
            assert abs(FH[q] - (simpson + L * (e * e) @ qv / 12)) < 1e-12


def test_sin_within_paper_bound_2d(orc):
    from test_oracle_mc_integrals import _exact_2d
    X = synth.uniform(50, 2, seed=73)
    cells = exact_cells(X, _fid)
    rowptr, col, A = _exact_csr(cells)
    T, C, _ = orc.vertices(X)
    _, _, IH, _ = orc.hmc(X, rowptr, col, A, T, C, ("sin_sq", 0))
    f2 = 6.0  # |d^2/dx^2 sin(x^2)| = |2 cos(x^2) - 4 x^2 sin(x^2)| <= 6 on [0, 1]
    total = 0.0
    for i, c in enumerate(cells):
        exact, _ = _exact_2d(c, X[i], lambda y: np.sin(y[:, 0] ** 2))
        P = np.concatenate(list(c["facet_pts"].values()))
        diam = max(np.linalg.norm(p - q) for p in P for q in P)
        assert abs(IH[i] - exact) <= c["volume"] * f2 * diam ** 2
        total += exact
    # the cells tile the square: sum of exact integrals = int_0^1 sin(x^2) dx
    from scipy import integrate
    assert abs(total - integrate.quad(lambda x: np.sin(x * x), 0, 1, epsabs=1e-14)[0]) < 1e-12
    assert abs(IH.sum() - total) < 0.01 * total
    # the exact areas' pyramid identity, as a check of the helper's facets
    for i, c in enumerate(cells):
        s = sum(facet_height(X, i, j, face_axis_side) * Ae for j, (Ae, _) in c["facets"].items())
        assert abs(s / 2 - c["volume"]) < 1e-12
