"""Brute-force references independent of the oracle's code.

* ``vertices_bruteforce``: every (d+1)-subset of nodes and box faces with at
  least one node and at most one face per axis; keep the subset iff its
  equidistant point (numpy.linalg.solve) lies in the box and no node is
  strictly closer than the subset's nodes (the incircle / empty-sphere
  criterion of Section 2.2).
* ``raycast_numpy``: the RayCast minimum written with numpy, formed as
  |x_j - v|^2 - |g - v|^2 over 2 u.(x_j - g) (Eq. (t)), a different rounding
  order than the oracle's.
"""
from __future__ import annotations

import itertools

import numpy as np


def face_id(a, s):
    return -(2 * a + s + 1)


def face_axis_side(gid):
    k = -gid - 1
    return k >> 1, k & 1


def vertices_bruteforce(X: np.ndarray, tol: float = 1e-10):
    N, d = X.shape
    gens = list(range(N)) + [face_id(a, s) for a in range(d) for s in (0, 1)]
    out = []
    for sub in itertools.combinations(gens, d + 1):
        nodes = [g for g in sub if g >= 0]
        faces = [g for g in sub if g < 0]
        if not nodes:
            continue
        axes = [face_axis_side(f)[0] for f in faces]
        if len(set(axes)) != len(axes):
            continue
        # rows: 2 (x_k - x_0) . r = |x_k|^2 - |x_0|^2 ; r_a = s
        Arows, brows = [], []
        x0 = X[nodes[0]]
        for k in nodes[1:]:
            Arows.append(2.0 * (X[k] - x0))
            brows.append(X[k] @ X[k] - x0 @ x0)
        for f in faces:
            a, s = face_axis_side(f)
            e = np.zeros(d)
            e[a] = 1.0
            Arows.append(e)
            brows.append(float(s))
        A = np.array(Arows)
        if abs(np.linalg.det(A)) < 1e-14:
            continue
        r = np.linalg.solve(A, np.array(brows))
        if np.any(r < -tol) or np.any(r > 1 + tol):
            continue
        R2 = np.sum((x0 - r) ** 2)
        dist2 = np.sum((X - r) ** 2, axis=1)
        others = np.setdiff1d(np.arange(N), nodes)
        if others.size and np.min(dist2[others]) < R2 * (1 - tol):
            continue
        out.append(tuple(sorted(sub)))
    return sorted(out)


def raycast_numpy(X, v, u, eta, box=True):
    N, d = X.shape
    g = X[eta[0]]
    num = np.sum((X - v) ** 2, axis=1) - np.sum((g - v) ** 2)
    den = (X - g) @ u
    t = np.full(N, np.inf)
    ok = den > 0
    ok[[e for e in eta if e >= 0]] = False
    t[ok] = num[ok] / (2.0 * den[ok])
    cands = [(t[j], 0, j, j) for j in range(N) if ok[j]]
    if box:
        for a in range(d):
            if u[a] < 0:
                cands.append(((0.0 - v[a]) / u[a], 1, 2 * a, face_id(a, 0)))
            elif u[a] > 0:
                cands.append(((1.0 - v[a]) / u[a], 1, 2 * a + 1, face_id(a, 1)))
    cands = [c for c in cands if c[3] not in eta]
    best = min(cands)
    return best[3], best[0]
