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
