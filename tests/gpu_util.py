"""Shared helpers of the GPU parity tests (inputs only, no method arithmetic)."""
import numpy as np
import pytest


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def random_unit(rng, n, d):
    u = rng.standard_normal((n, d))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def edge_rays(orc, X, tuples, coords, nmax, rng):
    """Rays of Algorithm 2: from oracle vertices along their edges."""
    d = X.shape[1]
    O, U, E = [], [], []
    for vid in rng.permutation(len(tuples)):
        sig = tuples[vid]
        for drop in range(d + 1):
            eta = [int(g) for q, g in enumerate(sig) if q != drop]
            nodes = sorted(g for g in eta if g >= 0)
            if not nodes:
                continue
            u = orc.search_direction(X, sig, drop)
            O.append(coords[vid])
            U.append(u)
            E.append([nodes[0]] + [g for g in eta if g != nodes[0]])
            if len(O) >= nmax:
                return np.array(O), np.array(U), np.array(E, np.int32)
    return np.array(O), np.array(U), np.array(E, np.int32)


def clustered_fan(R=256, n_cluster=40, seed=0):
    """Node g at (0.2, 0.5), a cluster of n_cluster nodes within 1e-9 of
    (0.62, 0.5) (one binary32 point, distinct binary64 points) and background
    nodes none of whose bisectors with g the fan of R rays from g (within
    3e-3 rad of +x) crosses before the cluster's: every ray keeps the whole
    cluster as binary32 candidates."""
    rng = np.random.default_rng(seed)
    g = np.array([0.2, 0.5])
    cl = np.array([0.62, 0.5]) + 1e-9 * rng.standard_normal((n_cluster, 2))
    bg = rng.uniform(0.0, 1.0, (600, 2))
    w = bg - g
    keep = (w[:, 0] <= 0) | (np.sum(w * w, axis=1) / (2 * np.maximum(w[:, 0] - 0.01 * np.abs(w[:, 1]), 1e-12)) > 0.3)
    X = np.vstack([g[None, :], cl, bg[keep]])
    th = rng.uniform(-3e-3, 3e-3, R)
    U = np.stack([np.cos(th), np.sin(th)], axis=1)
    return X, np.repeat(X[:1], R, axis=0), U, np.zeros((R, 1), np.int32)
