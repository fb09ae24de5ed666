"""Pins of the oracle on generic graphs (Sec. 2.2: D = I, A = the 0/1 adjacency)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import meshgen  # noqa: E402
import oracle  # noqa: E402


def csr_of(adj):
    n = len(adj)
    rowptr = np.zeros(n + 1, np.int32)
    col = []
    for i in range(n):
        js = sorted(adj[i])
        col += js
        rowptr[i + 1] = rowptr[i] + len(js)
    return rowptr, np.array(col, np.int32)


def test_path_biharmonic_closed_form():
    # path 0 - 1 - 2: L = V - A = [[1,-1,0],[-1,2,-1],[0,-1,1]] and M = L^2 with D = I
    rp, col = csr_of([[1], [0, 2], [1]])
    M = oracle.biharmonic(oracle.graph_operators(rp, col)).todense()
    assert np.array_equal(M, np.array([[2.0, -3.0, 1.0], [-3.0, 6.0, -3.0], [1.0, -3.0, 2.0]]))


def test_cycle_biharmonic_is_circulant():
    # cycle of 8: L = circulant(2, -1, ..., -1), so M = L^2 = circulant(6, -4, 1, 0, ..., 0, 1, -4)
    n = 8
    rp, col = csr_of([[(i - 1) % n, (i + 1) % n] for i in range(n)])
    M = oracle.biharmonic(oracle.graph_operators(rp, col)).todense()
    ref = np.zeros((n, n))
    for i in range(n):
        ref[i, i] = 6.0
        ref[i, (i + 1) % n] = ref[i, (i - 1) % n] = -4.0
        ref[i, (i + 2) % n] = ref[i, (i - 2) % n] = 1.0
    assert np.array_equal(M, ref)


def test_grid_graph_hop_distances_are_manhattan():
    nx, ny = 7, 5
    rp, col = meshgen.grid_graph(nx, ny)
    g = oracle.graph_operators(rp, col)
    src = np.array([0, 3 + nx * 2, nx * ny - 1], np.int32)
    D = oracle.geodesics(g, src)
    for a, s in enumerate(src):
        for v in range(nx * ny):
            assert D[a, v] == abs(v % nx - s % nx) + abs(v // nx - s // nx)


def test_knn_graph_operator_reproduces_constants_and_landmarks():
    rp, col, length, _ = meshgen.knn_graph(400, 6, seed=3)
    g = oracle.graph_operators(rp, col, length)
    idx, mind = oracle.fps(g, 25, 0)
    assert mind[idx].max() == 0.0 and mind.max() > 0.0 and np.unique(idx).size == 25
    P = oracle.interpolation(oracle.biharmonic(g), idx)
    assert np.array_equal(P[idx], np.eye(25))
    # M 1 = L (L 1) = 0: constants are biharmonic, so every row of P sums to one
    assert np.abs(P.sum(axis=1) - 1.0).max() < 1e-9
    # geodesics along the given lengths: an edge is never longer than its length
    D = oracle.geodesics(g, idx[:3])
    for a, s in enumerate(idx[:3]):
        for q in range(rp[s], rp[s + 1]):
            assert D[a, col[q]] <= length[q]
