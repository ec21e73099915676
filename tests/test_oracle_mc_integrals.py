"""Pins of the oracle's Monte Carlo function integrals (Section 3.1, Eqs.
mc-help1 and full_MC_integration, Algorithm 3): F_d over each boundary facet
and F_V over each cell, for f = 1, linear / quadratic polynomials and the
paper's sin(x_1^2), against exact integrals over the qhull cells (centroids
for linear f, Gauss-Legendre quadrature on the fan triangles and edges for
the rest) within a few standard errors, and F_d(f = 1) = A exactly."""
import numpy as np
import pytest
from scipy import stats

from exact_cells import exact_cells
from paper_2405_10050_gb300 import synth


def _fid(a, s):
    return -(2 * a + s + 1)


def _per_ray_terms(orc, X, R, seed, res, f, m):
    """Per-ray summands (scaled so that their mean over k is the estimate)
    of F_V (N x R) and of F_d (N x R, each ray's facet given by res.hit),
    for the standard errors only."""
    N, d = X.shape
    S = orc.sphere_area(d)
    U = orc.mc_directions(seed, 0, N, R, d)
    t = orc.mc_tsamples(seed, 0, N, R, m)
    l = res.l
    y = X[:, None, None, :] + (t * l[:, :, None])[..., None] * U[:, :, None, :]
    fy = orc.func_eval(f, y.reshape(-1, d)).reshape(N, R, m)
    cV = S * np.mean(fy * t ** (d - 1), axis=2) * l ** d
    r = X[:, None, :] + l[..., None] * U
    fr = orc.func_eval(f, r.reshape(-1, d)).reshape(N, R)
    a = np.empty((N, R))
    for i in range(N):
        for k in range(R):
            j = int(res.hit[i, k])
            if j >= 0:
                a[i, k] = 2 * l[i, k] ** d / np.linalg.norm(X[j] - X[i])
            else:
                ax = (-j - 1) >> 1
                a[i, k] = l[i, k] ** (d - 1) / abs(U[i, k, ax])
    return cV, S * fr * a


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


def _exact_2d(cell, xi, g, n=24):
    """Exact (to quadrature accuracy) integral of g over the polygon cell
    (fan triangles (x_i, p, q) in collapsed coordinates) and over each edge."""
    s, ws = _gl(n)
    vol = 0.0
    edges = {}
    for j, P in cell["facet_pts"].items():
        p, q = P[0], P[1]
        det = abs((p[0] - xi[0]) * (q[1] - xi[1]) - (p[1] - xi[1]) * (q[0] - xi[0]))
        S_, T_ = np.meshgrid(s, s, indexing="ij")
        pts = xi + S_[..., None] * ((1 - T_)[..., None] * (p - xi) + T_[..., None] * (q - xi))
        W = np.outer(ws, ws) * S_ * det
        vol += np.sum(W * g(pts.reshape(-1, 2)).reshape(W.shape))
        e = p + s[:, None] * (q - p)
        edges[j] = np.linalg.norm(q - p) * np.sum(ws * g(e))
    return vol, edges


def _check(FV, Fd, res, cV, cd, exact_vol, exact_facets, N, R, big=0.05):
    zs_v = []
    for i in range(N):
        se = np.std(cV[i]) / np.sqrt(R)
        zs_v.append((FV[i] - exact_vol[i]) / se)
    zs_v = np.array(zs_v)
    assert np.max(np.abs(zs_v)) < 5.0, np.max(np.abs(zs_v))
    assert abs(np.mean(zs_v)) < 5.0 / np.sqrt(N)
    zs_a = []
    for i in range(N):
        row = dict(zip(res.col[res.rowptr[i]:res.rowptr[i + 1]], range(res.rowptr[i], res.rowptr[i + 1])))
        tot = sum(abs(v[1]) for v in exact_facets[i].values())
        for j, (area, val) in exact_facets[i].items():
            if area > big * tot and j in row:
                contrib = np.where(res.hit[i] == j, cd[i], 0.0)
                se = np.std(contrib) / np.sqrt(R)
                if se == 0.0:  # f vanishes on the facet (sin(x_1^2) on x_1 = 0)
                    assert abs(Fd[row[j]] - val) < 1e-14
                    continue
                zs_a.append((Fd[row[j]] - val) / se)
    zs_a = np.array(zs_a)
    assert len(zs_a) > N
    assert np.max(np.abs(zs_a)) < 5.0, np.max(np.abs(zs_a))
    assert abs(np.mean(zs_a)) < 5.0 / np.sqrt(len(zs_a))


def test_tsamples_uniform_and_apart_from_directions(orc):
    """t_ks is U(0,1) (Kolmogorov-Smirnov), strictly inside (0,1), the mean of
    t^{d-1} is 1/d, and t is uncorrelated with the ray's direction."""
    t = orc.mc_tsamples(11, 0, 64, 256, 4)
    assert t.min() > 0.0 and t.max() < 1.0
    assert stats.kstest(t.ravel(), "uniform").pvalue > 1e-3
    for d in (2, 3, 5):
        assert abs(np.mean(t ** (d - 1)) - 1.0 / d) < 4 * np.std(t ** (d - 1)) / np.sqrt(t.size)
    U = orc.mc_directions(11, 0, 64, 256, 3)
    for a in range(3):
        r = np.corrcoef(t[:, :, 0].ravel(), U[:, :, a].ravel())[0, 1]
        assert abs(r) < 4.0 / np.sqrt(t[:, :, 0].size)


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_surface_integral_of_one_is_the_area(orc, d):
    """Algorithm 3: with f = 1 the facet integrals are the areas A_ij, term by
    term, so F_d = A bit for bit; F_V(f = 1) and V differ only by the t
    samples."""
    X = synth.uniform(40, d, seed=d + 30)
    R = 128
    res = orc.mc_integrate(X, R, seed=4)
    FV, Fd = orc.mc_integrals_all(X, R, 4, res, ("one",), 3)
    assert np.array_equal(Fd, res.A)
    assert np.all(FV > 0)


@pytest.mark.parametrize("d,N", [(2, 40), (3, 30)])
def test_linear_and_constant_f_match_exact_cells(orc, d, N):
    """f = 1 and f linear: the exact integrals are V (c0 + b.centroid) over
    the cell and A_ij (c0 + b.centroid_ij) over a facet (qhull cells); the
    estimates are within 5 standard errors, unbiased in aggregate."""
    X = synth.uniform(N, d, seed=40 + d)
    cells = exact_cells(X, _fid)
    R, m, seed = 4096, 2, 9
    res = orc.mc_integrate(X, R, seed=seed)
    for f in (("one",), ("poly2", 0.5, [3.0, -2.0, 1.5], [0.0, 0.0, 0.0])):
        c0 = 1.0 if f[0] == "one" else f[1]
        b = np.zeros(d) if f[0] == "one" else np.asarray(f[2][:d])
        FV, Fd = orc.mc_integrals_all(X, R, seed, res, f, m)
        cV, cd = _per_ray_terms(orc, X, R, seed, res, f, m)
        ev = [c["volume"] * (c0 + b @ c["centroid"]) for c in cells]
        ef = [{j: (A, A * (c0 + b @ cen)) for j, (A, cen) in c["facets"].items()} for c in cells]
        _check(FV, Fd, res, cV, cd, ev, ef, N, R)


def test_sin_and_quadratic_f_match_quadrature_2d(orc):
    """f = sin(x_1^2) (the integrand of the paper's Section 4) and a quadratic:
    exact integrals by Gauss-Legendre quadrature over each polygon's fan
    triangles and edges; estimates within 5 standard errors."""
    N, d = 40, 2
    X = synth.uniform(N, d, seed=77)
    cells = exact_cells(X, _fid)
    R, m, seed = 4096, 2, 13
    res = orc.mc_integrate(X, R, seed=seed)
    fs = [(("sin_sq", 0), lambda y: np.sin(y[:, 0] ** 2)),
          (("poly2", 0.2, [0.5, -1.0], [2.0, 1.0]), lambda y: 0.2 + 0.5 * y[:, 0] - y[:, 1] + 2 * y[:, 0] ** 2 + y[:, 1] ** 2)]
    for f, g in fs:
        FV, Fd = orc.mc_integrals_all(X, R, seed, res, f, m)
        cV, cd = _per_ray_terms(orc, X, R, seed, res, f, m)
        ev, ef = [], []
        for i, c in enumerate(cells):
            vol, edges = _exact_2d(c, X[i], g)
            ev.append(vol)
            ef.append({j: (c["facets"][j][0], edges[j]) for j in edges})
        _check(FV, Fd, res, cV, cd, ev, ef, N, R)


def test_quadrature_helper_on_known_integrals():
    """The quadrature itself: over the unit-square cell of a single node the
    integral of sin(x^2) is the Fresnel-type value from scipy's quad, and of
    x^2 + y^2 is 2/3; each edge integral of 1 is its length."""
    from scipy import integrate
    X = np.array([[0.3, 0.6]])
    cells = exact_cells(X, _fid)
    vol, edges = _exact_2d(cells[0], X[0], lambda y: np.sin(y[:, 0] ** 2))
    ref = integrate.quad(lambda x: np.sin(x * x), 0.0, 1.0, epsabs=1e-14)[0]
    assert abs(vol - ref) < 1e-13
    vol2, _ = _exact_2d(cells[0], X[0], lambda y: y[:, 0] ** 2 + y[:, 1] ** 2)
    assert abs(vol2 - 2.0 / 3.0) < 1e-13
    _, e1 = _exact_2d(cells[0], X[0], lambda y: np.ones(len(y)))
    assert all(abs(v - 1.0) < 1e-13 for v in e1.values())
