"""Brute-force references used to pin the oracle (tiny inputs only).

Nothing here calls the oracle: each function recomputes its quantity from the
mesh by the most direct route (all-edges relaxation, Floyd-Warshall, dense
matrices), so that a mistake in the oracle shows up as a disagreement.
"""
from __future__ import annotations

import math

import numpy as np


def edge_list(faces: np.ndarray) -> np.ndarray:
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]]).astype(np.int64)
    e.sort(axis=1)
    return np.unique(e, axis=0)


def edge_len_py(xyz: np.ndarray, i: int, j: int) -> float:
    """sqrt((dx*dx + dy*dy) + dz*dz) with dx = x_j - x_i, in Python floats (IEEE double, no FMA)."""
    dx = float(xyz[j, 0]) - float(xyz[i, 0])
    dy = float(xyz[j, 1]) - float(xyz[i, 1])
    dz = float(xyz[j, 2]) - float(xyz[i, 2])
    return math.sqrt((dx * dx + dy * dy) + dz * dz)


def bellman_ford(n: int, edges: np.ndarray, xyz: np.ndarray, src: int) -> np.ndarray:
    """Relax every directed edge until nothing changes; path lengths are left folds from src."""
    d = [math.inf] * n
    d[src] = 0.0
    arcs = []
    for a, b in edges:
        arcs.append((int(a), int(b), edge_len_py(xyz, int(a), int(b))))
        arcs.append((int(b), int(a), edge_len_py(xyz, int(b), int(a))))
    changed = True
    while changed:
        changed = False
        for a, b, w in arcs:
            if d[a] + w < d[b]:
                d[b] = d[a] + w
                changed = True
    return np.array(d)


def floyd_warshall(n: int, edges: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0.0)
    for a, b in edges:
        w = float(np.linalg.norm(xyz[a] - xyz[b]))
        D[a, b] = D[b, a] = min(D[a, b], w)
    for k in range(n):
        D = np.minimum(D, D[:, k : k + 1] + D[k : k + 1, :])
    return D


def fps_from_matrix(Dfull: np.ndarray, l: int, first: int) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 5 on a full distance matrix: argmax of the running minimum, lowest index on ties."""
    n = Dfull.shape[0]
    mind = np.full(n, np.inf)
    idx = []
    b = first
    for _ in range(l):
        idx.append(b)
        mind = np.minimum(mind, Dfull[b])
        b = int(np.argmax(mind))  # numpy returns the first maximum
    return np.array(idx), mind


def triangle_areas(xyz: np.ndarray, faces: np.ndarray) -> np.ndarray:
    a, b, c = xyz[faces[:, 0]], xyz[faces[:, 1]], xyz[faces[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def dense_laplacian(g) -> np.ndarray:
    """L = V - A from the oracle graph arrays, densely."""
    n = g.n
    A = np.zeros((n, n))
    for i in range(n):
        s, e = g.rowptr[i], g.rowptr[i + 1]
        A[i, g.col[s:e]] = g.A[s:e]
    return np.diag(A.sum(axis=1)) - A


def procrustes_residual(X: np.ndarray, Y: np.ndarray) -> float:
    """min over rotations/reflections R of ||Xc R - Yc||_F / ||Yc||_F (both centred)."""
    Xc = X - X.mean(axis=0)
    Yc = Y - Y.mean(axis=0)
    U, _, Vt = np.linalg.svd(Xc.T @ Yc)
    R = U @ Vt
    return float(np.linalg.norm(Xc @ R - Yc) / np.linalg.norm(Yc))
