"""Exact clipped Voronoi cells from scipy's qhull (independent of the oracle).

For node i, its cell is the intersection of the halfspaces
2 (x_j - x_i) . y <= |x_j|^2 - |x_i|^2 (j != i) with the unit box; qhull's
HalfspaceIntersection gives its vertices and, per vertex, the halfspaces that
meet there, from which every facet (one per neighbour or box face) is read
off.  Volumes, facet areas and facet centroids follow from a fan
triangulation.  Used to pin the Monte Carlo oracle (Section 3.1) and its
adjoint; the pyramid identity V_i = (1/d) sum_j h_ij A_ij (Section 3.2)
checks this helper itself.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import ConvexHull, HalfspaceIntersection


def _polygon_area_centroid_3d(P):
    c0 = P.mean(axis=0)
    # order the facet's vertices by angle around c0 in the facet plane
    _, _, vt = np.linalg.svd(P - c0)
    e1, e2 = vt[0], vt[1]
    ang = np.arctan2((P - c0) @ e2, (P - c0) @ e1)
    Q = P[np.argsort(ang)]
    area, cen = 0.0, np.zeros(3)
    for k in range(1, len(Q) - 1):
        a = 0.5 * np.linalg.norm(np.cross(Q[k] - Q[0], Q[k + 1] - Q[0]))
        area += a
        cen += a * (Q[0] + Q[k] + Q[k + 1]) / 3.0
    return area, cen / area


def exact_cells(X: np.ndarray, face_id):
    """Per cell i: dict(volume=..., facets={gen_id: (area, centroid)},
    facet_pts={gen_id: the facet's vertices (d = 2: its two end points)},
    centroid=the cell's centroid)."""
    N, d = X.shape
    assert d in (2, 3)
    cells = []
    for i in range(N):
        others = np.delete(np.arange(N), i)
        W = X[others] - X[i]
        # halfspace rows [A | b] with A y + b <= 0
        A_nodes = 2.0 * W
        b_nodes = -(np.sum(X[others] ** 2, axis=1) - np.sum(X[i] ** 2))
        A_box = np.vstack([-np.eye(d), np.eye(d)])
        b_box = np.concatenate([np.zeros(d), -np.ones(d)])
        H = np.vstack([np.column_stack([A_nodes, b_nodes]), np.column_stack([A_box, b_box])])
        ids = list(others) + [face_id(a, 0) for a in range(d)] + [face_id(a, 1) for a in range(d)]
        hs = HalfspaceIntersection(H, X[i].copy())
        verts = hs.intersections
        vol = ConvexHull(verts).volume
        facets = {}
        facet_pts = {}
        dual = hs.dual_facets
        for h in range(H.shape[0]):
            on = [v for v in range(len(verts)) if h in dual[v]]
            if len(on) < d:
                continue
            P = verts[on]
            if d == 2:
                P = np.unique(np.round(P, 14), axis=0)
                if len(P) < 2:
                    continue
                length = np.linalg.norm(P.max(axis=0) - P.min(axis=0))
                if length < 1e-14:
                    continue
                facets[int(ids[h])] = (length, P.mean(axis=0))
                facet_pts[int(ids[h])] = P[[np.argmin(P @ (P[-1] - P[0])), np.argmax(P @ (P[-1] - P[0]))]]
            else:
                if len(P) < 3:
                    continue
                area, cen = _polygon_area_centroid_3d(P)
                if area < 1e-14:
                    continue
                facets[int(ids[h])] = (area, cen)
                facet_pts[int(ids[h])] = P
        cells.append({"volume": vol, "facets": facets, "facet_pts": facet_pts,
                      "centroid": _fan_centroid(verts, X[i])})
    return cells


def _fan_centroid(verts, p0):
    """Centroid of the convex hull of verts, from simplices fanned out of the
    interior point p0 over the hull's boundary facets."""
    d = verts.shape[1]
    hull = ConvexHull(verts)
    vol, cen = 0.0, np.zeros(d)
    for simp in hull.simplices:
        P = verts[simp]
        v = abs(np.linalg.det(P - p0)) / float(np.prod(np.arange(1, d + 1)))
        vol += v
        cen += v * (P.sum(axis=0) + p0) / (d + 1)
    return cen / vol


def facet_height(X, i, gid, face_axis_side):
    """Distance from x_i to the facet's plane: |x_j - x_i|/2 or the face."""
    if gid >= 0:
        return 0.5 * np.linalg.norm(X[gid] - X[i])
    a, s = face_axis_side(gid)
    return X[i, a] if s == 0 else 1.0 - X[i, a]


def exact_volume_gradient(X, cells):
    """dV_i/dx_k by the transport of the bisector planes (a Reynolds-type
    identity): dV_i/dx_j = A_ij (x_j - c_ij)/|x_j - x_i| for a neighbour j,
    dV_i/dx_i = sum_j A_ij (c_ij - x_i)/|x_j - x_i|; box faces do not move.
    Returns G[i, k, :] = dV_i/dx_k."""
    N, d = X.shape
    G = np.zeros((N, N, d))
    for i, c in enumerate(cells):
        for j, (A, cen) in c["facets"].items():
            if j < 0:
                continue
            r = np.linalg.norm(X[j] - X[i])
            G[i, j] += A * (X[j] - cen) / r
            G[i, i] += A * (cen - X[i]) / r
    return G
