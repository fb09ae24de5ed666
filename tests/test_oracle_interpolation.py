"""Pins for the oracle's interpolation operator P = [I; -M_uu^{-1} M_ub] (Eq. 3, Eq. 6) and thresholding (Eq. 8)."""
import numpy as np
import pytest

import meshgen
import oracle


def _setup(m, l, first=0):
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, l, first)
    M = oracle.biharmonic(g)
    return g, idx, M


@pytest.fixture(scope="module")
def cases():
    out = []
    for m, l in ((meshgen.icosphere(3, noise=0.01, seed=0), 32), (meshgen.torus(30, 24, seed=1), 36),
                 (meshgen.sphere_patch_bumps(24), 20)):
        g, idx, M = _setup(m, l)
        out.append((m, g, idx, M, oracle.interpolation(M, idx)))
    return out


def test_landmark_rows_are_identity_bitwise(cases):
    for m, g, idx, M, P in cases:
        assert np.array_equal(P[idx], np.eye(idx.size))


def test_rows_sum_to_one(cases):
    # M 1 = 0, so the constant function is biharmonic and interpolating ones gives ones.
    for m, g, idx, M, P in cases:
        assert np.abs(P.sum(axis=1) - 1.0).max() < 1e-10


def test_columns_solve_the_biharmonic_system(cases):
    for m, g, idx, M, P in cases:
        Md = M.todense()
        unk = np.setdiff1d(np.arange(m.n), idx)
        Muu, Mub = Md[np.ix_(unk, unk)], Md[np.ix_(unk, idx)]
        res = Muu @ P[unk] + Mub
        assert np.linalg.norm(res) < 1e-12 * np.linalg.norm(Mub)
        ref = np.linalg.solve(Muu, -Mub)
        assert np.abs(P[unk] - ref).max() < 1e-10


def test_selected_columns_match_full_solve(cases):
    m, g, idx, M, P = cases[1]
    cols = np.array([5, 0, 17], np.int32)
    Pc = oracle.interpolation(M, idx, cols)
    assert np.array_equal(Pc, P[:, cols])


def test_all_vertices_as_landmarks_gives_identity():
    # l = n: P -> I and the approximation P W P^T equals the distance matrix exactly (Sec. 3.1).
    m = meshgen.icosphere(1, noise=0.01, seed=2)
    g, idx, M = _setup(m, m.n)
    P = oracle.interpolation(M, idx)
    # column j of P is the indicator of vertex idx[j]
    for j in range(m.n):
        col = np.zeros(m.n)
        col[idx[j]] = 1.0
        assert np.array_equal(P[:, j], col)
    W = oracle.landmark_block(g, idx)
    K = oracle.geodesics(g, np.arange(m.n))
    Kt = P @ W @ P.T
    Ksym = 0.5 * (K + K.T)
    np.fill_diagonal(Ksym, 0.0)
    assert np.array_equal(Kt, Ksym)


def _brute_rows(P, idx, p_row):
    n, l = P.shape
    keep = min(p_row, l)
    out = {}
    lm = {int(b): j for j, b in enumerate(idx)}
    for i in range(n):
        if i in lm:
            out[i] = [(lm[i], 1.0)]
            continue
        cand = sorted(range(l), key=lambda j: (-abs(P[i, j]), j))[:keep]
        out[i] = [(j, P[i, j]) for j in sorted(cand)]
    return out


def test_sparsify_rows_brute_force_with_ties():
    rng = np.random.default_rng(0)
    n, l = 40, 9
    idx = np.array([3, 7, 11, 19, 23, 29, 31, 37, 0])
    P = rng.normal(size=(n, l))
    P[np.abs(P) < 0.4] = 0.25 * np.sign(P[np.abs(P) < 0.4] + 1e-9)  # many exact magnitude ties
    P[idx] = np.eye(l)
    for p_row in (1, 3, 9, 20):
        S = oracle.sparsify_rows(P, idx, p_row)
        ref = _brute_rows(P, idx, p_row)
        assert S.rowptr[-1] == l + (n - l) * min(p_row, l)
        for i in range(n):
            got = list(zip(S.col[S.rowptr[i] : S.rowptr[i + 1]].tolist(), S.val[S.rowptr[i] : S.rowptr[i + 1]].tolist()))
            assert got == ref[i]


def test_sparsify_cols_brute_force():
    rng = np.random.default_rng(1)
    n, l = 50, 6
    idx = np.array([1, 9, 17, 25, 33, 41])
    P = rng.normal(size=(n, l))
    P[::7] = np.round(P[::7], 1)  # some ties
    P[idx] = np.eye(l)
    p_row = 3
    p = oracle.column_mode_p(n, l, p_row)
    assert p == round((n - l) * p_row / l + 1e-12)
    S = oracle.sparsify_cols(P, idx, p_row).todense()
    unk = [i for i in range(n) if i not in set(idx.tolist())]
    for j in range(l):
        cand = sorted(unk, key=lambda i: (-abs(P[i, j]), i))[:p]
        want = np.zeros(n)
        want[cand] = P[cand, j]
        want[idx[j]] = 1.0
        assert np.array_equal(S[:, j], want)


def test_column_mode_p_rounding():
    assert oracle.column_mode_p(642, 32, 8) == 153  # (610 * 8) / 32 = 152.5 -> 153 (half up)
    assert oracle.column_mode_p(50000, 500, 16) == 1584
    assert oracle.column_mode_p(10, 9, 1) == 1


def test_interpolation_is_the_exactly_rounded_solution():
    """Eq. 3 solved to the last bit: the oracle's columns of P_u against a 30-digit solve (mpmath LU)
    of the same system.  At cond(M_uu) ~ 4e4 a plain FP64 factorisation is off by ~1e-13 of the
    column's largest entry; with iterative refinement on a double-double residual the oracle is
    within one rounding of the exact solution."""
    mpmath = pytest.importorskip("mpmath")
    m = meshgen.torus(14, 10, 1.0, 0.3, 0.2, seed=7)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 6, 0)
    M = oracle.biharmonic(g)
    cols = np.array([0, 3], np.int32)
    P = oracle.interpolation(M, idx, cols)
    Md = M.todense()
    unk = np.setdiff1d(np.arange(m.n), idx)
    Muu = Md[np.ix_(unk, unk)]
    assert np.linalg.cond(Muu) > 1e4  # hard enough that an unrefined solve misses the bar
    mpmath.mp.dps = 30
    A = mpmath.matrix(Muu.tolist())
    for c, j in enumerate(cols):
        b = mpmath.matrix((-Md[unk, idx[j]]).tolist())
        exact = np.array([float(v) for v in mpmath.lu_solve(A, b)])
        err = np.abs(P[unk, c] - exact).max() / np.abs(exact).max()
        assert err <= 2 * np.finfo(float).eps, f"column {j}: {err:.2e}"
