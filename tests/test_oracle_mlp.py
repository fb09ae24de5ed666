"""Pins for the oracle's warm-start network: BF16 rounding and backpropagation."""
import numpy as np
import pytest

import oracle


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.normal(size=4096) * 10.0 ** rng.uniform(-6, 6, 4096)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.bf16_round(x), ref)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(40, oracle.MLP_F))
    T = rng.normal(size=40)
    p = rng.normal(size=oracle.MLP_PARAMS) * 0.2
    loss, g = oracle.mlp_loss_grad_f64(X, T, p)
    for i in rng.choice(oracle.MLP_PARAMS, 60, replace=False).tolist() + [oracle.MLP_PARAMS - 1, 0, 384, 448]:
        e = np.zeros_like(p)
        h = 1e-6
        e[i] = h
        fd = (oracle.mlp_loss_grad_f64(X, T, p + e)[0] - oracle.mlp_loss_grad_f64(X, T, p - e)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_zero_network_is_constant_prediction():
    # all weights zero except b3: y = b3 for every sample, so the loss is mean (b3 - t)^2
    X = np.ones((5, oracle.MLP_F))
    T = np.arange(5.0)
    p = np.zeros(oracle.MLP_PARAMS)
    p[-1] = 2.0
    loss, g = oracle.mlp_loss_grad_f64(X, T, p)
    assert loss == np.mean((2.0 - T) ** 2)
    assert g[-1] == pytest.approx(np.mean(2 * (2.0 - T)))
    assert np.all(g[:-65] == 0.0)


# ---------------------------------------------------------------- learned preconditioner

def _pinned_laplacian(level=2, l=12):
    """L_uu of an icosphere (cotangent Laplacian with the FPS landmarks removed), CSR with diagonal."""
    import scipy.sparse as sp
    import meshgen
    m = meshgen.icosphere(level, 0.01, 0)
    g = oracle.mesh_operators(m.xyz, m.faces)
    n = g.n
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    A = sp.csr_matrix((g.A, (rows, g.col)), shape=(n, n))
    L = (sp.diags(np.asarray(A.sum(1)).ravel()) - A).tocsr()
    idx, _ = oracle.fps(g, l, 0)
    u = np.setdiff1d(np.arange(n), idx)
    Luu = L[u][:, u].tocsr()
    Luu.sort_indices()
    Aub = A[u][:, idx].toarray()
    return Luu, Aub


def _dense_jacobi_loss(Luu, B):
    A = Luu.toarray()
    Dinv = np.diag(1.0 / np.diag(A))
    loss = 0.0
    for c in range(B.shape[1]):
        b = B[:, c]
        if not b.any():
            continue
        r = A @ (Dinv @ b) - b
        loss += (r @ r) / (B.shape[1] * (b @ b))
    return loss


def test_precond_features_closed_form():
    # 3x3 SPD matrix with a full pattern: every feature written out by hand
    A = np.array([[4.0, -1.0, 0.5], [-1.0, 5.0, -2.0], [0.5, -2.0, 6.0]])
    rowptr = np.array([0, 3, 6, 9])
    col = np.array([0, 1, 2] * 3)
    val = A.ravel()
    feat, rows, d = oracle.precond_features(rowptr, col, val)
    leak = [(4 - 1.5) / 4, (5 - 3) / 5, (6 - 2.5) / 6]
    for e in range(9):
        i, j = divmod(e, 3)
        want = [1.0 if i == j else 0.0, 0.0 if i == j else -A[i, j] / A[i, i], 0.0 if i == j else -A[i, j] / A[j, j],
                leak[i], leak[j], 3 / 7]
        np.testing.assert_allclose(feat[e], np.float32(want), rtol=0, atol=0)


def test_precond_zero_output_is_jacobi():
    rng = np.random.default_rng(3)
    Luu, Aub = _pinned_laplacian()
    p = rng.normal(size=oracle.MLP_PARAMS) * 0.3
    p[-65:] = 0.0  # w3, b3: network output 0, G = D^{-1/2}
    B = Aub[:, :8]
    loss, _ = oracle.precond_loss_grad_f64(Luu.indptr, Luu.indices, Luu.data, B, p)
    assert loss == pytest.approx(_dense_jacobi_loss(Luu, B), rel=1e-12)
    G = oracle.precond_factor(Luu.indptr, Luu.indices, Luu.data, p).toarray()
    np.testing.assert_allclose(G, np.diag(1.0 / np.sqrt(Luu.diagonal())), rtol=0, atol=0)


def test_precond_diagonal_matrix_exact_at_jacobi():
    # Jacobi inverts a diagonal matrix exactly: zero loss and zero gradient at the Jacobi start
    m = 10
    rowptr = np.arange(m + 1)
    col = np.arange(m)
    val = np.linspace(1.0, 5.0, m)
    p = np.random.default_rng(4).normal(size=oracle.MLP_PARAMS) * 0.3
    p[-65:] = 0.0
    B = np.random.default_rng(5).normal(size=(m, 3))
    loss, g = oracle.precond_loss_grad_f64(rowptr, col, val, B, p)
    assert loss < 1e-28
    assert np.abs(g).max() < 1e-12


def test_precond_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    Luu, Aub = _pinned_laplacian()
    B = np.concatenate([Aub[:, :5], rng.normal(size=(Aub.shape[0], 2))], axis=1)
    p = rng.normal(size=oracle.MLP_PARAMS) * 0.2
    args = (Luu.indptr, Luu.indices, Luu.data, B)
    loss, g = oracle.precond_loss_grad_f64(*args, p)
    picks = rng.choice(oracle.MLP_PARAMS, 40, replace=False).tolist() + [0, 5, 384, 448, 4544, 4608, 4672]
    for i in picks:
        e = np.zeros_like(p)
        h = 1e-6
        e[i] = h
        fd = (oracle.precond_loss_grad_f64(*args, p + e)[0] - oracle.precond_loss_grad_f64(*args, p - e)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])), (i, fd, g[i])


def test_precond_loss_is_residual_of_one_application():
    # the loss equals the mean relative squared residual of x = G^T G b, computed densely
    rng = np.random.default_rng(7)
    Luu, Aub = _pinned_laplacian()
    p = rng.normal(size=oracle.MLP_PARAMS) * 0.2
    B = Aub[:, :6]
    loss, _ = oracle.precond_loss_grad_f64(Luu.indptr, Luu.indices, Luu.data, B, p)
    G = oracle.precond_factor(Luu.indptr, Luu.indices, Luu.data, p).toarray()
    A = Luu.toarray()
    want = np.mean([np.sum((A @ G.T @ G @ B[:, c] - B[:, c]) ** 2) / np.sum(B[:, c] ** 2) for c in range(6)])
    assert loss == pytest.approx(want, rel=1e-12)


def test_precond_pairs_with_exact_solutions_equal_residual_form():
    # with x_c the exact solution of A x_c = b_c, ||A (M b - x)|| = ||A M b - b||
    import scipy.sparse.linalg as sla
    rng = np.random.default_rng(8)
    Luu, Aub = _pinned_laplacian()
    B = Aub[:, :5]
    X = sla.splu(Luu.tocsc()).solve(B)
    p = rng.normal(size=oracle.MLP_PARAMS) * 0.2
    l0, g0 = oracle.precond_loss_grad_f64(Luu.indptr, Luu.indices, Luu.data, B, p)
    l1, g1 = oracle.precond_loss_grad_f64(Luu.indptr, Luu.indices, Luu.data, B, p, X)
    assert l1 == pytest.approx(l0, rel=1e-9)
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-9 * np.abs(g0).max())
    # an inexact solution shifts the target: the loss then differs
    l2, _ = oracle.precond_loss_grad_f64(Luu.indptr, Luu.indices, Luu.data, B, p, X * 1.01)
    assert abs(l2 - l0) > 1e-6 * l0
