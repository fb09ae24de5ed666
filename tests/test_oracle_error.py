"""Pins of oracle.bha_error, the relative error of K~ = P W P^T (Eq. 9) as the paper measures it
(Sec. 4.1: eps = ||K~ - K||_F^2 / ||K||_F^2, estimated on sampled rows for large meshes)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import meshgen  # noqa: E402
import oracle  # noqa: E402


def csr(dense):
    dense = np.asarray(dense, dtype=np.float64)
    rp, cols, vals = [0], [], []
    for r in dense:
        nz = np.nonzero(r)[0]
        cols += nz.tolist()
        vals += r[nz].tolist()
        rp.append(len(cols))
    return oracle.CSR(np.array(rp, np.int32), np.array(cols, np.int32), np.array(vals), dense.shape[1])


# A path a - c - b with unit edges and landmarks a, b; the middle vertex c interpolates both with
# weight 1/2.  Worked by hand:
#   K = [[0,2,1],[2,0,1],[1,1,0]],  W = [[0,2],[2,0]],  P = [[1,0],[0,1],[.5,.5]]
#   P W = [[0,2],[2,0],[1,1]],  K~ = P W P^T = [[0,2,1],[2,0,1],[1,1,1]]
#   K~ - K is 1 at (c, c) only: num = 1, den = ||K||^2 = 12.
#   squared: P (W.W) P^T = [[0,4,2],[4,0,2],[2,2,2]] against K.K = [[0,4,1],[4,0,1],[1,1,0]]:
#   differences 1, 1 (rows a, b at column c), 1, 1, 2 (row c): num = 8, den = 36.
PATH_K = np.array([[0.0, 2.0, 1.0], [2.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
PATH_W = np.array([[0.0, 2.0], [2.0, 0.0]])
PATH_P = csr([[1.0, 0.0], [0.0, 1.0], [0.5, 0.5]])


def test_path_by_hand():
    num, den = oracle.bha_error(PATH_P, PATH_W, np.arange(3), PATH_K)
    assert (num, den) == (1.0, 12.0)
    num, den = oracle.bha_error(PATH_P, PATH_W, np.arange(3), PATH_K, squared=True)
    assert (num, den) == (8.0, 36.0)


def test_path_sampled_rows():
    # row c alone: K~_c = [1,1,1] vs K_c = [1,1,0] -> (1, 2); rows a, b alone: exact -> (0, 5) each
    assert oracle.bha_error(PATH_P, PATH_W, np.array([2]), PATH_K[[2]]) == (1.0, 2.0)
    assert oracle.bha_error(PATH_P, PATH_W, np.array([0, 1]), PATH_K[[0, 1]]) == (0.0, 10.0)


def test_zero_approximation_is_error_one():
    K = np.abs(np.random.default_rng(0).normal(size=(5, 5)))
    P = csr(np.ones((5, 1)))
    num, den = oracle.bha_error(P, np.zeros((1, 1)), np.arange(5), K)
    assert num == den
    # a constant approximation: sum of (c - K)^2 written out
    num, _ = oracle.bha_error(P, np.array([[0.75]]), np.arange(5), K)
    ref = sum((0.75 - K[i, j]) ** 2 for i in range(5) for j in range(5))
    assert abs(num - ref) <= 1e-14 * ref


def test_every_vertex_a_landmark_is_exact():
    # l = n: P is the identity up to the landmark order, so K~ = K and the error is exactly 0
    m = meshgen.icosphere(1, noise=0.02, seed=3)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, m.n, 0)
    P = oracle.sparsify_rows(oracle.interpolation(oracle.biharmonic(g), idx), idx, 4)
    W = oracle.landmark_block(g, idx)
    K = np.zeros((m.n, m.n))
    K[np.ix_(idx, idx)] = W
    rows = np.array([0, 5, 17, m.n - 1])
    num, den = oracle.bha_error(P, W, rows, K[rows])
    assert num == 0.0 and den == np.sum(K[rows] ** 2)


def test_sampled_estimate_matches_the_full_error_in_expectation():
    # the row-sample estimate is unbiased: averaging num/den-weighted samples over all rows
    # recovers the full ratio exactly when every row is taken once
    m = meshgen.torus(16, 12, 1.0, 0.3, 0.2, seed=4)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 20, 0)
    P = oracle.sparsify_rows(oracle.interpolation(oracle.biharmonic(g), idx), idx, 6)
    W = oracle.landmark_block(g, idx)
    K = oracle.geodesics(g, np.arange(m.n, dtype=np.int32))
    full = oracle.bha_error(P, W, np.arange(m.n), K)
    parts = [oracle.bha_error(P, W, np.arange(a, min(a + 50, m.n)), K[a:a + 50]) for a in range(0, m.n, 50)]
    assert abs(sum(p[0] for p in parts) - full[0]) <= 1e-12 * full[0]
    assert abs(sum(p[1] for p in parts) - full[1]) <= 1e-12 * full[1]
    assert 0.0 < full[0] / full[1] < 0.1  # 20 landmarks on 192 vertices: a rough but useful approximation


def test_exact_sphere_distances_are_interpolated_with_small_falling_error():
    """The operator's accuracy on a surface with known distances: interpolating the exact great-circle
    landmark distances of a unit sphere reproduces the whole great-circle matrix with an error that
    falls steadily as landmarks are added (measured 1.2e-3, 3.1e-4, 8.3e-5, 2.8e-5 at l = 16 ... 128)."""
    s = meshgen.icosphere(3)
    g = oracle.mesh_operators(s.xyz, s.faces)
    K = np.arccos(np.clip(s.xyz @ s.xyz.T, -1.0, 1.0))
    M = oracle.biharmonic(g)
    eps = []
    for l in (16, 32, 64, 128):
        idx, _ = oracle.fps(g, l, 0)
        P = oracle.sparsify_rows(oracle.interpolation(M, idx), idx, min(l, 50))
        num, den = oracle.bha_error(P, K[np.ix_(idx, idx)], np.arange(s.n), K)
        eps.append(num / den)
    assert eps[0] < 2e-3 and all(b < 0.5 * a for a, b in zip(eps, eps[1:]))
