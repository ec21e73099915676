"""Seeded synthetic node sets (the only module shared by the tests, the
benchmark and the smoke check).  It holds none of the method's arithmetic:
it only draws points.

Recipes (Section 4 of the paper uses iid uniform nodes in the unit cube; the
mixtures follow the high-dimensional and batched workloads):

* ``uniform(N, d, seed)``: iid U[0,1]^d, numpy PCG64 seeded with ``seed``.
* ``gaussian_mixture(N, d, K, sigma, seed)``: K centres iid U[0,1]^d, each
  point picks a centre uniformly and adds N(0, sigma^2 I); points outside the
  cube are rejected and redrawn (clamping would put nodes exactly on faces).
* ``batch_sets(nsets, seed)``: set s has N = floor(exp(U(ln 200, ln 20000))),
  d uniform in {2..8}; the first half uniform, the second half 8-component
  mixtures with sigma 0.05.
"""
from __future__ import annotations

import math

import numpy as np


def uniform(N: int, d: int, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).random((N, d))


def gaussian_mixture(N: int, d: int, K: int, sigma: float, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    centres = rng.random((K, d))
    out = np.empty((0, d))
    while out.shape[0] < N:
        m = max(2 * (N - out.shape[0]), 1024)
        lab = rng.integers(0, K, size=m)
        pts = centres[lab] + sigma * rng.standard_normal((m, d))
        ok = np.all((pts > 0.0) & (pts < 1.0), axis=1)
        out = np.concatenate([out, pts[ok]], axis=0)
    return np.ascontiguousarray(out[:N])


def batch_sets(nsets: int = 512, seed: int = 0, n_lo: int = 200, n_hi: int = 20000):
    """List of (X, d) for the batched workload; set s uses seed (seed, s)."""
    sets = []
    for s in range(nsets):
        rng = np.random.default_rng([seed, s])
        N = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.integers(2, 9))
        if s < nsets // 2:
            X = uniform(N, d, seed=int(rng.integers(0, 2**31)))
        else:
            X = gaussian_mixture(N, d, 8, 0.05, seed=int(rng.integers(0, 2**31)))
        sets.append((X, d))
    return sets
