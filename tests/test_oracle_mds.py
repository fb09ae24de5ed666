"""Pins for the oracle's eigensolver and classical-scaling routes (Eq. 4, Sec. 3.3)."""
import json
import math
import os

import numpy as np
import pytest

import meshgen
import oracle
from tests import _brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_jacobi_two_by_two_closed_form():
    for a, b, d in ((2.0, 1.0, 3.0), (1.0, -4.0, 1.0), (5.0, 1e-9, 5.0), (-1.0, 2.0, 7.0)):
        w, V = oracle.jacobi_eigh(np.array([[a, b], [b, d]]))
        mid, rad = (a + d) / 2, math.hypot((a - d) / 2, b)
        np.testing.assert_allclose(w, [mid + rad, mid - rad], rtol=1e-14, atol=1e-15 * abs(mid))


def test_jacobi_diagonal_and_path_laplacian():
    w, V = oracle.jacobi_eigh(np.diag([3.0, -1.0, 2.0, 0.5]))
    assert np.array_equal(w, [3.0, 2.0, 0.5, -1.0])
    n = 17
    L = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    L[0, 0] = L[-1, -1] = 1.0  # path graph Laplacian: eigenvalues 2 - 2 cos(k pi / n)
    w, V = oracle.jacobi_eigh(L)
    want = np.sort(2 - 2 * np.cos(np.arange(n) * np.pi / n))[::-1]
    np.testing.assert_allclose(w, want, atol=1e-13)


def test_jacobi_random_symmetric():
    rng = np.random.default_rng(0)
    for m in (5, 40, 97):
        X = rng.normal(size=(m, m))
        S = X + X.T
        w, V = oracle.jacobi_eigh(S)
        np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(S))[::-1], atol=1e-12 * np.abs(w).max())
        np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-13)
        np.testing.assert_allclose(S @ V, V * w, atol=1e-12 * np.abs(w).max())


def test_classical_mds_recovers_euclidean_points():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(60, 3)) * [3.0, 2.0, 1.0]
    E = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    Z, theta = oracle.mds_full(E, 3)
    assert _brute.procrustes_residual(Z, X) < 1e-12
    Xc = X - X.mean(0)
    np.testing.assert_allclose(theta, np.linalg.svd(Xc, compute_uv=False) ** 2, rtol=1e-12)


def _csr_identity(n, idx):
    # P with column j = indicator of vertex idx[j]
    col = np.zeros(n, np.int32)
    col[idx] = np.arange(n)
    return oracle.CSR(np.arange(n + 1, dtype=np.int32), col, np.ones(n), n)


def test_all_landmarks_low_rank_equals_full_mds():
    m = meshgen.icosphere(2, noise=0.01, seed=5)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, m.n, 0)
    W = oracle.landmark_block(g, idx)
    Z, theta = oracle.mds_gram(_csr_identity(m.n, idx), W, 3)
    K = oracle.geodesics(g, np.arange(m.n))
    K = 0.5 * (K + K.T)
    np.fill_diagonal(K, 0.0)
    Zf, thf = oracle.mds_full(K * K, 3)
    np.testing.assert_allclose(theta, thf, rtol=1e-10)
    np.testing.assert_allclose(Z @ Z.T, Zf @ Zf.T, atol=1e-9 * thf[0])


@pytest.fixture(scope="module")
def c1():
    m, w = meshgen.workload("icosphere3_l32")
    return m, w, oracle.sbmds(m.xyz, m.faces, w["l"], w["p_row"], w["k"], w["first"])


def test_gram_route_equals_qr_route(c1):
    m, w, r = c1
    Zq, thq = oracle.mds_qr(r.P.todense(), r.W, 3)
    np.testing.assert_allclose(r.theta, thq, rtol=1e-10)
    np.testing.assert_allclose(r.Z @ r.Z.T, Zq @ Zq.T, atol=1e-10 * thq[0])
    # also on the dense operator (where G is singular along the ones vector)
    Pd = oracle.CSR(*_dense_to_csr(r.P_dense), r.W.shape[0])
    Zg, thg = oracle.mds_gram(Pd, r.W, 3)
    Zq, thq = oracle.mds_qr(r.P_dense, r.W, 3)
    np.testing.assert_allclose(thg, thq, rtol=1e-10)


def _dense_to_csr(D):
    rp, cols, vals = [0], [], []
    for row in D:
        nz = np.nonzero(row)[0]
        cols.append(nz)
        vals.append(row[nz])
        rp.append(rp[-1] + nz.size)
    return np.array(rp, np.int32), np.concatenate(cols).astype(np.int32), np.concatenate(vals)


def test_gram_is_centred_and_column_sums(c1):
    m, w, r = c1
    c, G = oracle.gram(r.P)
    Pd = r.P.todense()
    np.testing.assert_allclose(c, Pd.sum(0), rtol=1e-14)
    JP = Pd - Pd.mean(0)
    np.testing.assert_allclose(G, JP.T @ JP, atol=1e-12 * np.abs(G).max())
    # dense P: J P 1 = 0, so G is singular along the ones vector
    cd, Gd = oracle.gram(oracle.CSR(*_dense_to_csr(r.P_dense), r.W.shape[0]))
    assert np.abs(Gd @ np.ones(Gd.shape[0])).max() < 1e-10 * np.abs(Gd).max()


def test_stress_eckart_young(c1):
    # With E~ = P (W.W) P^T and B = -1/2 J E~ J, the rank-k scaling leaves
    # ||Z Z^T - B||_F^2 = sum of the squared eigenvalues outside the top k.
    m, w, r = c1
    Pd = r.P.todense()
    Et = Pd @ (r.W * r.W) @ Pd.T
    n = m.n
    J = np.eye(n) - 1.0 / n
    B = -0.5 * J @ Et @ J
    lam = np.sort(np.linalg.eigvalsh(0.5 * (B + B.T)))[::-1]
    np.testing.assert_allclose(lam[:3], r.theta, rtol=1e-10)
    lhs = np.linalg.norm(r.Z @ r.Z.T - B) ** 2
    rhs = np.sum(lam[3:] ** 2)
    assert abs(lhs - rhs) < 1e-9 * np.sum(lam**2)
    s = oracle.stress(r.Z, Et)
    assert abs(s - math.sqrt(rhs / np.sum(lam**2))) < 1e-9


def test_flat_grid_embedding_is_near_isometric():
    # On a flat, jittered grid the scaling of interpolated squared Euclidean landmark
    # distances recovers the grid up to a rigid motion (residual from the open boundary,
    # measured 0.027); with mesh-edge distances the low-rank embedding stays close to the
    # full classical scaling of the same edge metric (which is itself anisotropic).
    m = meshgen.flat_grid(30, 24, jitter=0.1, seed=3)
    X = m.xyz[:, :2]
    r = oracle.sbmds(m.xyz, m.faces, 60, 16, 2, 0)
    Eu = np.sqrt(((X[:, None] - X[None]) ** 2).sum(-1))
    Z, _ = oracle.mds_gram(r.P, Eu[np.ix_(r.idx, r.idx)], 2)
    assert _brute.procrustes_residual(Z, X) < 0.04
    K = oracle.geodesics(r.graph, np.arange(m.n))
    K = 0.5 * (K + K.T)
    Zf, _ = oracle.mds_full(K * K, 2)
    assert _brute.procrustes_residual(r.Z, Zf) < 0.05


def test_operator_reproduces_great_circle_distances():
    # Interpolating exact great-circle landmark distances on a fine unit sphere reproduces
    # great-circle distances elsewhere, with the error measure of Sec. 4.1.  The dense
    # operator's error falls as l grows; thresholding error falls as p_row grows and is
    # indistinguishable from the dense operator at p_row = 50 (the paper's Sec. 4.1 finding
    # that sBHA at p_row 50..100 matches BHA).  Values measured: dense l=120 1.95e-5,
    # l=240 5.8e-6; rows kept 8/16/32/50: 1.2e-2, 1.2e-3, 3.3e-5, 2.0e-5.
    m = meshgen.icosphere(4)
    g = oracle.mesh_operators(m.xyz, m.faces)
    M = oracle.biharmonic(g)
    gc = np.arccos(np.clip(m.xyz @ m.xyz.T, -1.0, 1.0))

    def eps(P, idx):
        Kt = P @ gc[np.ix_(idx, idx)] @ P.T
        return np.linalg.norm(Kt - gc) ** 2 / np.linalg.norm(gc) ** 2

    dense = {}
    for l in (120, 240):
        idx, _ = oracle.fps(g, l, 0)
        Pd = oracle.interpolation(M, idx)
        dense[l] = eps(Pd, idx)
    assert dense[120] < 5e-5 and dense[240] < 0.5 * dense[120]
    idx, _ = oracle.fps(g, 120, 0)
    Pd = oracle.interpolation(M, idx)
    sparse = [eps(oracle.sparsify_rows(Pd, idx, p).todense(), idx) for p in (8, 16, 32, 50)]
    assert all(a > b for a, b in zip(sparse, sparse[1:]))
    assert sparse[-1] < 1.05 * dense[120]


def test_paper_memory_figures():
    # The paper's full-matrix figure for its 1.8M-vertex mesh is n^2 doubles (Sec. 4.3, Fig. 1).
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as f:
        gold = json.load(f)
    d = gold["dragon1800k"]
    full_bytes = d["n"] ** 2 * 8
    assert abs(full_bytes / 1e12 - d["full_matrix_TB"]) < 0.1
    # the approximation is W (l^2 doubles) plus the sparse operator; W alone is 20.0 GB
    w_bytes = d["l"] ** 2 * 8
    assert w_bytes / 1e9 < d["approx_GB"] < w_bytes / 1e9 + d["n"] * 50 * 12 / 1e9
