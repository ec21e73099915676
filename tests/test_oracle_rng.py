"""Pins of the oracle's direction generator (Section 3.1: uniform directions
from a normalised Gaussian draw) against things other than itself."""
import ctypes
import os

import numpy as np
import pytest
from scipy import stats


def _curand():
    for p in ["/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"]:
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator(orc):
    """Philox4x32-10 against NVIDIA's independent host implementation
    (curandCreateGeneratorHost, PHILOX4_32_10): curand lays block b of the
    output on counter (b >> 16, 0, b & 0xffff, 0) with key (seed lo, seed hi)."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        for seed in [0, 0x123456789ABCDEF0, 7]:
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(0)) == 0
            n = 1 << 19
            out = np.zeros(n, np.uint32)
            assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
            b = np.arange(n // 4)
            ctr = np.zeros((n // 4, 4), np.uint32)
            ctr[:, 0] = b >> 16
            ctr[:, 2] = b & 0xFFFF
            mine = orc.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32]).reshape(-1)
            assert np.array_equal(mine, out)
    finally:
        cr.curandDestroyGenerator(gen)


def test_log32_against_libm(orc):
    rng = np.random.default_rng(1)
    x = np.concatenate([
        ((rng.integers(0, 2**23, 200000) * 2 + 1) * 2.0**-24).astype(np.float32),
        np.float32(2.0) ** -np.arange(0, 24, dtype=np.float32),
        np.nextafter(np.float32(np.sqrt(2) / 2), np.float32(0)) * np.float32(2.0) ** -np.arange(0, 20, dtype=np.float32),
        np.array([1.0, 0.5, 0.70710677, 0.7071068, 1.0 - 2**-24, 2**-24], np.float32),
    ])
    y = orc.log32(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    err = np.abs(y - ref)
    # a few binary32 ulps of the result (|ln x| <= 17 here)
    assert np.all(err <= 4 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) + 1e-30)
    assert orc.log32(np.array([1.0], np.float32))[0] == 0.0


def test_sincos_all_24bit_angles(orc):
    a = np.arange(1 << 24, dtype=np.uint32)
    c, s = orc.sincos2pi24(a)
    ang = 2.0 * np.pi * a.astype(np.float64) / 2.0**24
    assert np.max(np.abs(c - np.cos(ang))) < 3e-7
    assert np.max(np.abs(s - np.sin(ang))) < 3e-7
    # octant boundaries are exact where the series gives exact values
    assert c[0] == 1.0 and s[0] == 0.0
    assert s[1 << 22] == 1.0 and c[1 << 23] == -1.0 and s[3 << 22] == -1.0


def test_direction_components_are_zero_or_above_5e_12(orc):
    """Every component of an MC direction (d <= 16) is 0 or above 5e-12 in
    magnitude, over every input the draw can take: the binary32 radius
    sqrt(-2 ln U) lies in [3.4e-4, 5.77] over all 2^23 values of U, the
    cosine and sine of all 2^24 angles are 0 or at least 3.7e-7 in
    magnitude, and |z| <= 4 * 5.77 at d = 16.  So a component rounds to 0 in
    binary32 only when it is 0 (the MC kernels' binary32 face tests rely on
    this)."""
    U = (np.arange(1 << 23, dtype=np.uint64) * 2 + 1).astype(np.float32) * np.float32(2.0**-24)
    L = orc.log32(U)
    assert np.all(L < 0)
    r = np.sqrt(np.float32(-2.0) * L)  # binary32, as in the draw
    assert r.min() >= 3.4e-4 and r.max() <= 5.77
    c, s = orc.sincos2pi24(np.arange(1 << 24, dtype=np.uint32))
    for v in (c, s):
        assert np.abs(v[v != 0]).min() >= 3.7e-7
    z_min = 3.4e-4 * 3.7e-7 * (1 - 2.0**-23)  # the product rounded in binary32
    assert z_min / (4 * 5.77 * (1 + 2.0**-50)) > 5e-12
    u = orc.mc_directions(seed=7, set_id=0, N=64, R=1024, d=16)
    assert np.abs(u[u != 0]).min() > 5e-12


def test_gaussian_draw_is_standard_normal(orc):
    z = orc.mc_gaussians32(seed=11, set_id=0, N=2000, R=64, d=4).reshape(-1).astype(np.float64)
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 5 * np.sqrt(24.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4


@pytest.mark.parametrize("d", [1, 2, 3, 5, 16])
def test_directions_uniform_on_sphere(orc, d):
    u = orc.mc_directions(seed=3, set_id=0, N=400, R=128, d=d).reshape(-1, d)
    n = u.shape[0]
    assert np.max(np.abs(np.linalg.norm(u, axis=1) - 1.0)) < 4e-16 * np.sqrt(d) + 1e-16
    assert np.all(np.abs(u.mean(axis=0)) < 5 / np.sqrt(n * d) + 1e-12)
    C = u.T @ u / n
    assert np.max(np.abs(C - np.eye(d) / d)) < 6 * np.sqrt(2.0 / n) / d + 1e-3 / d
    if d == 1:
        assert np.all(np.abs(np.abs(u) - 1.0) <= 2.3e-16)  # +-1 up to one rounding
        assert abs((u > 0).mean() - 0.5) < 5 * 0.5 / np.sqrt(n)
    if d == 3:  # Archimedes: each coordinate of a uniform point on S^2 is U[-1,1]
        assert stats.kstest(u[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-4


def test_direction_streams_are_distinct(orc):
    a = orc.mc_directions(5, 0, 50, 8, 3)
    b = orc.mc_directions(6, 0, 50, 8, 3)
    c = orc.mc_directions(5, 1, 50, 8, 3)
    assert len(np.unique(a.reshape(-1, 3), axis=0)) == 400
    assert not np.any(np.all(a == b, axis=2)) and not np.any(np.all(a == c, axis=2))
