"""Plain FP64 CPU oracle for sparse biharmonic MDS (arXiv:1705.10887).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library: the numerics live in ``sbha_oracle.c`` (built by
``build()`` with ``-ffp-contract=off``) and in the numpy glue below, which uses
only library primitives (sort, matmul, QR, a sparse LU solve, a dense solve) as single steps.

Readings of the paper that the oracle fixes (each stated where it is used):
  * geodesics are shortest paths along mesh edges with Euclidean edge lengths;
  * farthest-point ties go to the lowest vertex index, b_1 = ``first``;
  * sparsification keeps, per non-landmark row, the min(p_row, l) entries of
    largest magnitude (ties: smaller column) -- or, in column mode (the literal
    Eq. 8), per column the p = round((n-l) p_row / l) entries of largest
    magnitude (ties: smaller row); landmark rows stay the identity;
  * the scaling step works on W (.) W, the squared landmark distances;
  * eigenvector signs: the largest-magnitude entry of each embedding column is
    made positive.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbha_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ENOTSPD, ORC_ENOCONV = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``sbha_oracle.c`` into ``liboracle.so`` (plain gcc, OpenMP if present)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11", "-o", _LIB, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        lib.orc_mesh_operators.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.orc_dijkstra.argtypes = [i64, vp, vp, vp, i32, vp]
        lib.orc_geodesics.argtypes = [i64, vp, vp, vp, vp, i32, vp, i32, vp]
        lib.orc_fps.argtypes = [i64, vp, vp, vp, i32, i32, vp, vp]
        lib.orc_weight_sums.argtypes = [i64, vp, vp, vp]
        lib.orc_biharmonic_nnz.argtypes = [i64, vp, vp, vp]
        lib.orc_biharmonic.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
        lib.orc_interpolation.argtypes = [i64, vp, vp, vp, vp, i32, vp, i32, vp]
        lib.orc_gram.argtypes = [i64, i32, vp, vp, vp, vp, vp]
        lib.orc_jacobi_eig.argtypes = [i32, vp, vp, vp, i32, ctypes.c_double]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(status: int, what: str):
    if status != ORC_OK:
        raise OracleError(f"{what}: oracle status {status}")


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


@dataclass
class Graph:
    """Edge graph of a mesh with its per-edge length and cotangent weight, and lumped mass."""

    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray  # int32 [nnz]
    length: np.ndarray  # float64 [nnz]
    A: np.ndarray  # float64 [nnz]
    D: np.ndarray  # float64 [n]

    @property
    def n(self) -> int:
        return self.rowptr.size - 1


def mesh_operators(xyz: np.ndarray, faces: np.ndarray) -> Graph:
    """Edge graph, edge lengths, cotangent adjacency A and lumped mass D (Sec. 2.2)."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    faces = np.ascontiguousarray(faces, dtype=np.int32)
    n, f = xyz.shape[0], faces.shape[0]
    rowptr = np.zeros(n + 1, np.int32)
    col = np.zeros(6 * f + 1, np.int32)
    length = np.zeros(6 * f + 1)
    A = np.zeros(6 * f + 1)
    D = np.zeros(n)
    nnz = ctypes.c_int64(0)
    _check(lib.orc_mesh_operators(n, f, _p(xyz), _p(faces), _p(rowptr), _p(col), _p(length), _p(A), _p(D),
                                  ctypes.byref(nnz)), "mesh_operators")
    e = nnz.value
    return Graph(rowptr, col[:e].copy(), length[:e].copy(), A[:e].copy(), D)


def weight_sums(g: Graph) -> np.ndarray:
    """V = diag of the row sums of A (Sec. 2.2), each summed left to right in column order."""
    V = np.zeros(g.n)
    _check(_load().orc_weight_sums(g.n, _p(g.rowptr), _p(g.A), _p(V)), "weight_sums")
    return V


def graph_operators(rowptr: np.ndarray, col: np.ndarray, length=None) -> Graph:
    """A generic graph as the paper treats it (Sec. 2.2): D = I and A = the 0/1 adjacency; the edges
    keep the given lengths (or 1) for the geodesics."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    nnz = col.size
    ln = np.ones(nnz) if length is None else np.ascontiguousarray(length, dtype=np.float64)
    return Graph(rowptr, col, ln, np.ones(nnz), np.ones(rowptr.size - 1))


def dijkstra(g: Graph, src: int) -> np.ndarray:
    """Shortest mesh-edge path length from ``src`` to every vertex (Eq. 1 on the edge graph)."""
    dist = np.zeros(g.n)
    _check(_load().orc_dijkstra(g.n, _p(g.rowptr), _p(g.col), _p(g.length), int(src), _p(dist)), "dijkstra")
    return dist


def geodesics(g: Graph, sources, targets=None) -> np.ndarray:
    """Distances, row-major (len(sources), len(targets) or n)."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    if targets is None:
        out = np.zeros((src.size, g.n))
        tp, t = None, 0
    else:
        tgt = np.ascontiguousarray(targets, dtype=np.int32)
        out = np.zeros((src.size, tgt.size))
        tp, t = _p(tgt), tgt.size
    _check(_load().orc_geodesics(g.n, _p(g.rowptr), _p(g.col), _p(g.length), _p(src), src.size, tp, t, _p(out)),
           "geodesics")
    return out


def fps(g: Graph, l: int, first: int = 0):
    """Farthest-point landmarks (Eq. 5).  Returns (idx int32[l], mind float64[n])."""
    idx = np.zeros(l, np.int32)
    mind = np.zeros(g.n)
    _check(_load().orc_fps(g.n, _p(g.rowptr), _p(g.col), _p(g.length), int(l), int(first), _p(idx), _p(mind)), "fps")
    return idx, mind


def landmark_block(g: Graph, idx: np.ndarray) -> np.ndarray:
    """W_ij = d(b_i, b_j) (Sec. 3), symmetrised as (W + W^T)/2 with a zero diagonal.

    Distances from b_i evaluated at b_j and from b_j at b_i are left folds along
    opposite directions of the path and may differ in the last bit; the mean of
    the two is the symmetric reading of the paper's symmetric d.
    """
    W = geodesics(g, idx, idx)
    W = (W + W.T) * 0.5
    np.fill_diagonal(W, 0.0)
    return W


@dataclass
class CSR:
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    ncols: int

    @property
    def nrows(self) -> int:
        return self.rowptr.size - 1

    def todense(self) -> np.ndarray:
        out = np.zeros((self.nrows, self.ncols))
        for i in range(self.nrows):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            out[i, self.col[s:e]] = self.val[s:e]
        return out


def biharmonic(g: Graph) -> CSR:
    """M = (V - A)^T D^{-1} (V - A) (Sec. 2.2) as CSR with the 2-ring pattern."""
    lib = _load()
    nnz = ctypes.c_int64(0)
    _check(lib.orc_biharmonic_nnz(g.n, _p(g.rowptr), _p(g.col), ctypes.byref(nnz)), "biharmonic_nnz")
    rp = np.zeros(g.n + 1, np.int32)
    col = np.zeros(nnz.value, np.int32)
    val = np.zeros(nnz.value)
    _check(lib.orc_biharmonic(g.n, _p(g.rowptr), _p(g.col), _p(g.A), _p(g.D), _p(rp), _p(col), _p(val)), "biharmonic")
    return CSR(rp, col, val, g.n)


def interpolation(M: CSR, idx: np.ndarray, cols=None) -> np.ndarray:
    """Dense columns of P = [I_l; -M_uu^{-1} M_ub] (Eq. 6) in vertex order, shape (n, len(cols)).

    Solved by envelope Cholesky of M_uu in reverse Cuthill-McKee order.
    """
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    l = idx.size
    cols = np.arange(l, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros((M.nrows, cols.size))
    _check(_load().orc_interpolation(M.nrows, _p(M.rowptr), _p(M.col), _p(M.val), _p(idx), l, _p(cols), cols.size,
                                     _p(out)), "interpolation")
    return out


def column_mode_p(n: int, l: int, p_row: int) -> int:
    """p = (n - l) p_row / l (Sec. 3.1), rounded half up, clamped to [1, n - l]."""
    p = ((n - l) * p_row * 2 + l) // (2 * l)
    return int(max(1, min(n - l, p)))


def sparsify_rows(P: np.ndarray, idx: np.ndarray, p_row: int) -> CSR:
    """Thresholding by rows: each non-landmark row keeps its min(p_row, l) largest |P_ij|.

    Ties in magnitude go to the smaller column.  Landmark rows are e_j.  Kept
    entries are stored in ascending column order.
    """
    n, l = P.shape
    is_lm = np.zeros(n, bool)
    is_lm[idx] = True
    lm_col = np.full(n, -1)
    lm_col[idx] = np.arange(l)
    keep = min(p_row, l)
    rowptr = np.zeros(n + 1, np.int64)
    cols, vals = [], []
    for i in range(n):
        if is_lm[i]:
            c = np.array([lm_col[i]])
            v = np.array([1.0])
        else:
            order = np.lexsort((np.arange(l), -np.abs(P[i])))  # |v| desc, then column asc
            c = np.sort(order[:keep])
            v = P[i, c]
        cols.append(c)
        vals.append(v)
        rowptr[i + 1] = rowptr[i] + c.size
    return CSR(rowptr.astype(np.int32), np.concatenate(cols).astype(np.int32), np.concatenate(vals), l)


def sparsify_cols(P: np.ndarray, idx: np.ndarray, p_row: int) -> CSR:
    """Thresholding by columns (Eq. 8 read literally): each column keeps its p largest |P_ij|
    over non-landmark rows, p = round((n - l) p_row / l); ties go to the smaller row."""
    n, l = P.shape
    p = column_mode_p(n, l, p_row)
    is_lm = np.zeros(n, bool)
    is_lm[idx] = True
    unk = np.nonzero(~is_lm)[0]
    mask = np.zeros((n, l), bool)
    for j in range(l):
        v = P[unk, j]
        order = np.lexsort((unk, -np.abs(v)))
        mask[unk[order[:p]], j] = True
    mask[idx, np.arange(l)] = True
    S = np.where(mask, P, 0.0)
    S[idx] = 0.0
    S[idx, np.arange(l)] = 1.0
    rowptr = np.zeros(n + 1, np.int64)
    cols, vals = [], []
    for i in range(n):
        c = np.nonzero(mask[i])[0] if not is_lm[i] else np.nonzero(S[i])[0]
        cols.append(c)
        vals.append(S[i, c])
        rowptr[i + 1] = rowptr[i] + c.size
    return CSR(rowptr.astype(np.int32), np.concatenate(cols).astype(np.int32), np.concatenate(vals), l)


def gram(P: CSR):
    """c = P^T 1 and G = (J P)^T (J P) = P^T P - c c^T / n (Sec. 3.3)."""
    n, l = P.nrows, P.ncols
    c = np.zeros(l)
    G = np.zeros((l, l))
    _check(_load().orc_gram(n, l, _p(P.rowptr), _p(P.col), _p(P.val), _p(c), _p(G)), "gram")
    return c, G


def jacobi_eigh(S: np.ndarray, max_sweeps: int = 100, tol: float = 1e-15):
    """Eigenpairs of a symmetric matrix by cyclic Jacobi, sorted by decreasing eigenvalue."""
    m = S.shape[0]
    A = np.ascontiguousarray(S, dtype=np.float64).copy()
    w = np.zeros(m)
    V = np.zeros((m, m))
    _check(_load().orc_jacobi_eig(m, _p(A), _p(w), _p(V), int(max_sweeps), float(tol)), "jacobi_eig")
    order = np.argsort(-w, kind="stable")
    return w[order], V[:, order]


def _sign_fix(Z: np.ndarray) -> np.ndarray:
    """Make the largest-magnitude entry of each column positive (first such entry on ties)."""
    Z = Z.copy()
    for c in range(Z.shape[1]):
        r = int(np.argmax(np.abs(Z[:, c])))
        if Z[r, c] < 0:
            Z[:, c] = -Z[:, c]
    return Z


def mds_gram(P: CSR, W: np.ndarray, k: int, rank_tol: float = 1e-12):
    """Low-rank classical scaling of -1/2 J P (W.W) P^T J (Sec. 3.3) through the Gram matrix.

    With G = (JP)^T (JP) = U S U^T (Jacobi), R = S^{1/2} U^T is a valid QR factor of
    J P (any R with R^T R = G differs from the QR one by an orthogonal factor, which
    leaves the eigenvalues and Z unchanged).  Eigenvalues S_i <= rank_tol * S_max
    are dropped (J P 1 = 0 for a dense P, so G is singular).  Then
    B = -1/2 R WE R^T = V Lam V^T (Jacobi), and
    Z = J P U S^{-1/2} V_k Lam_k^{1/2} = Q V_k Lam_k^{1/2}, Lam^{1/2} of max(theta, 0).
    Returns (Z (n, k), theta (k)).
    """
    n = P.nrows
    c, G = gram(P)
    s, U = jacobi_eigh(G)
    r = int(np.sum(s > rank_tol * s[0]))
    s, U = s[:r], U[:, :r]
    R = np.sqrt(s)[:, None] * U.T
    WE = W * W
    B = -0.5 * (R @ WE @ R.T)
    B = 0.5 * (B + B.T)
    theta, V = jacobi_eigh(B)
    theta_k, V_k = theta[:k], V[:, :k]
    T = U @ (V_k / np.sqrt(s)[:, None]) * np.sqrt(np.maximum(theta_k, 0.0))[None, :]
    PT = P_times(P, T)
    Z = PT - (c @ T)[None, :] / n
    return _sign_fix(Z), theta_k


def P_times(P: CSR, T: np.ndarray) -> np.ndarray:
    out = np.zeros((P.nrows, T.shape[1]))
    for i in range(P.nrows):
        s, e = P.rowptr[i], P.rowptr[i + 1]
        out[i] = P.val[s:e] @ T[P.col[s:e]]
    return out


def mds_qr(P_dense: np.ndarray, W: np.ndarray, k: int):
    """The paper's literal route (Sec. 3.3): Q R = J P, eig of -1/2 R W R^T, Z = Q V_k Lam_k^{1/2}.

    Uses squared landmark distances W.W.  Returns (Z, theta_k)."""
    n = P_dense.shape[0]
    JP = P_dense - P_dense.mean(axis=0, keepdims=True)
    Q, R = np.linalg.qr(JP)
    B = -0.5 * (R @ (W * W) @ R.T)
    B = 0.5 * (B + B.T)
    theta, V = jacobi_eigh(B)
    Z = Q @ V[:, :k] * np.sqrt(np.maximum(theta[:k], 0.0))[None, :]
    return _sign_fix(Z), theta[:k]


def mds_full(E: np.ndarray, k: int):
    """Classical MDS (Eq. 4): eig of -1/2 J E J, Z = V_k Lam_k^{1/2}.  E = squared distances."""
    n = E.shape[0]
    J = np.eye(n) - np.ones((n, n)) / n
    B = -0.5 * (J @ E @ J)
    B = 0.5 * (B + B.T)
    theta, V = jacobi_eigh(B)
    Z = V[:, :k] * np.sqrt(np.maximum(theta[:k], 0.0))[None, :]
    return _sign_fix(Z), theta[:k]


def stress(Z: np.ndarray, E: np.ndarray) -> float:
    """Normalised stress || Z Z^T + 1/2 J E J ||_F / || 1/2 J E J ||_F (Eq. 4's objective)."""
    n = E.shape[0]
    Ec = E - E.mean(axis=0, keepdims=True)
    Ec = Ec - Ec.mean(axis=1, keepdims=True)
    half = 0.5 * Ec
    Zc = Z - Z.mean(axis=0, keepdims=True)
    return float(np.linalg.norm(Zc @ Zc.T + half) / np.linalg.norm(half))


def heat_geodesics(xyz: np.ndarray, faces: np.ndarray, sources, m: float = 1.0) -> np.ndarray:
    """Approximate geodesic distances by the heat method (the distances the paper's experiments use,
    Sec. 4, after Crane et al. 2013), one row per source:

      1. u = (D + t L)^{-1} delta_s, the heat after time t = m h^2 (h the mean edge length; L = V - A
         and D from Sec. 2.2, so D + t L is the backward Euler step of du/dt = -D^{-1} L u);
      2. on every triangle the unit field X = -grad u / |grad u| of the linear interpolant of u;
      3. the integrated divergence of X at each vertex, 1/2 sum over its triangles of
         cot(angle opposite e1) (e1 . X) + cot(angle opposite e2) (e2 . X), e1 and e2 the two edges
         leaving the vertex;
      4. phi with L phi = -div X (L is minus the cotangent Laplacian), fixed by phi(s) = 0.

    The linear solves are scipy's sparse LU (a library primitive); the rest is written out here.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    g = mesh_operators(xyz, faces)
    n = g.n
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    A = sp.csr_matrix((g.A, (rows, g.col)), shape=(n, n))
    L = (sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A).tocsc()
    h = float(np.mean(g.length))
    t = m * h * h
    H = (sp.diags(g.D) + t * L).tocsc()
    a, b, c = faces[:, 0], faces[:, 1], faces[:, 2]
    xa, xb, xc = xyz[a], xyz[b], xyz[c]
    nrm = np.cross(xb - xa, xc - xa)
    twice_area = np.linalg.norm(nrm, axis=1)
    N = nrm / twice_area[:, None]

    def cot(p, q, r):  # cotangent of the angle at r between r->p and r->q
        u, v = p - r, q - r
        return np.sum(u * v, axis=1) / np.linalg.norm(np.cross(u, v), axis=1)

    cot_a, cot_b, cot_c = cot(xb, xc, xa), cot(xc, xa, xb), cot(xa, xb, xc)
    out = np.zeros((len(sources), n))
    for k, s in enumerate(np.asarray(sources)):
        delta = np.zeros(n)
        delta[s] = 1.0
        u = spl.spsolve(H, delta)
        # grad u = 1/(2 area) sum_i u_i N x e_i, e_i the edge opposite vertex i, counter-clockwise
        grad = (u[a][:, None] * np.cross(N, xc - xb) + u[b][:, None] * np.cross(N, xa - xc)
                + u[c][:, None] * np.cross(N, xb - xa)) / twice_area[:, None]
        gn = np.linalg.norm(grad, axis=1)
        X = np.where(gn[:, None] > 0, -grad / np.where(gn > 0, gn, 1.0)[:, None], 0.0)
        div = np.zeros(n)
        np.add.at(div, a, 0.5 * (cot_c * np.sum((xb - xa) * X, axis=1) + cot_b * np.sum((xc - xa) * X, axis=1)))
        np.add.at(div, b, 0.5 * (cot_a * np.sum((xc - xb) * X, axis=1) + cot_c * np.sum((xa - xb) * X, axis=1)))
        np.add.at(div, c, 0.5 * (cot_b * np.sum((xa - xc) * X, axis=1) + cot_a * np.sum((xb - xc) * X, axis=1)))
        keep = np.setdiff1d(np.arange(n), [s])
        phi = np.zeros(n)
        phi[keep] = spl.spsolve(L[keep][:, keep].tocsc(), -div[keep])
        out[k] = phi
    return out


def fmds_interpolation(M: CSR, idx: np.ndarray, P: np.ndarray, mu: float) -> np.ndarray:
    """The FMDS interpolation matrix from the biharmonic one (Sec. 3.4.2): H = P (M_bb + mu I + M_bu P_u)^{-1} mu.

    P is the dense n x l operator of Eq. 6 (landmark rows e_j), M the biharmonic operator; H lets the
    landmark values deviate by an amount that mu controls.  The l x l solve is numpy's (a library
    primitive)."""
    idx = np.asarray(idx)
    Md = M.todense()
    unk = np.setdiff1d(np.arange(M.nrows), idx)
    S = Md[np.ix_(idx, idx)] + mu * np.eye(idx.size) + Md[np.ix_(idx, unk)] @ P[unk]
    return P @ np.linalg.solve(S, mu * np.eye(idx.size))


def bha_error(P: CSR, W: np.ndarray, rows: np.ndarray, K_rows: np.ndarray, squared: bool = False):
    """Relative error of the approximation K~ = P W P^T (Eq. 9) on sampled rows (Sec. 4.1).

    The paper measures eps = ||K~ - K||_F^2 / ||K||_F^2 and, when K is too large to hold,
    estimates it on a random subset of rows.  For the rows S (K_rows[i] = exact row rows[i] of K)
    this returns (num, den) = (sum over S of ||K~_s - K_s||^2, sum over S of ||K_s||^2), so
    eps ~= num / den, exact when S is every row.  squared=True compares the squared distances
    K (.) K with P (W (.) W) P^T, the matrix that classical scaling factors.
    """
    rows = np.asarray(rows)
    Pd = P.todense()
    Wm = W * W if squared else W
    Km = K_rows * K_rows if squared else K_rows
    Kt = Pd[rows] @ Wm @ Pd.T
    return float(np.sum((Kt - Km) ** 2)), float(np.sum(Km ** 2))


@dataclass
class Result:
    graph: Graph
    idx: np.ndarray
    mind: np.ndarray
    W: np.ndarray
    M: CSR
    P_dense: np.ndarray
    P: CSR
    Z: np.ndarray
    theta: np.ndarray


def sbmds(xyz: np.ndarray, faces: np.ndarray, l: int, p_row: int, k: int = 3, first: int = 0,
          mode: str = "row") -> Result:
    """The whole pipeline, stage by stage in the paper's order (Sec. 3 - 3.3)."""
    g = mesh_operators(xyz, faces)
    idx, mind = fps(g, l, first)
    W = landmark_block(g, idx)
    M = biharmonic(g)
    Pd = interpolation(M, idx)
    P = sparsify_rows(Pd, idx, p_row) if mode == "row" else sparsify_cols(Pd, idx, p_row)
    Z, theta = mds_gram(P, W, k)
    return Result(g, idx, mind, W, M, Pd, P, Z, theta)


# ----------------------------------------------------------------------------
# Warm-start network: y(x) = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3, parameters
# stored in BF16 (round to nearest even), loss = mean (y - t)^2.  Plain FP64 backprop.

MLP_H, MLP_F = 64, 6
MLP_PARAMS = MLP_H * MLP_F + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _mlp_split(p):
    H, F = MLP_H, MLP_F
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def _mlp_forward(X, p):
    W1, b1, W2, b2, w3, b3 = _mlp_split(p)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h1, h2, h2 @ w3 + b3


def _mlp_backward(X, h1, h2, dy, p):
    """Gradient of sum_s dy_s y(x_s) with respect to the parameters (back-propagation)."""
    W1, b1, W2, b2, w3, b3 = _mlp_split(p)
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    d2 = dy[:, None] * w3[None, :] * (1.0 - h2 ** 2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 ** 2)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def mlp_loss_grad_f64(X, T, p):
    """Loss and gradient with respect to the FP64 parameter vector p (no rounding)."""
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    p = np.asarray(p, np.float64)
    h1, h2, y = _mlp_forward(X, p)
    err = y - T
    return float(np.mean(err ** 2)), _mlp_backward(X, h1, h2, 2.0 * err / X.shape[0], p)


def mlp_loss_grad(X, T, params):
    """The network's loss and gradient as the library defines them: parameters rounded to BF16 first."""
    return mlp_loss_grad_f64(X, T, bf16_round(params))


# ----------------------------------------------------------------------------
# Learned preconditioner M^{-1} = G^T G of an SPD matrix A (CSR, symmetric pattern, diagonal
# present): G on A's pattern, G_ij = (delta_ij + y(f_ij)) / sqrt(A_ii), features
#   f_ij = [i == j, -A_ij / A_ii, -A_ij / A_jj, leak_i, leak_j, nnz(row i) / 7],
#   leak_i = (A_ii - sum_{k != i} |A_ik|) / A_ii,
# training loss  sum_c ||A (G^T G b_c - x_c)||^2 / (ncols ||b_c||^2) over (b_c, x_c) with A x_c = b_c.

def precond_features(rowptr, col, val):
    """(features float32 [nnz, 6], row of each entry, diagonal of each row)."""
    rowptr = np.asarray(rowptr, np.int64)
    col = np.asarray(col, np.int64)
    val = np.asarray(val, np.float64)
    m = rowptr.size - 1
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    isd = rows == col
    d = np.zeros(m)
    d[rows[isd]] = val[isd]
    off = np.bincount(rows[~isd], weights=np.abs(val[~isd]), minlength=m)
    leak = (d - off) / d
    feat = np.zeros((col.size, 6))
    feat[:, 0] = isd
    feat[:, 1] = np.where(isd, 0.0, -val / d[rows])
    feat[:, 2] = np.where(isd, 0.0, -val / d[col])
    feat[:, 3] = leak[rows]
    feat[:, 4] = leak[col]
    feat[:, 5] = np.diff(rowptr)[rows] / 7.0
    return feat.astype(np.float32), rows, d


def precond_factor(rowptr, col, val, p):
    """G (scipy CSR) for the FP64 parameter vector p."""
    import scipy.sparse as sp
    feat, rows, d = precond_features(rowptr, col, val)
    _, _, y = _mlp_forward(feat.astype(np.float64), np.asarray(p, np.float64))
    g = ((rows == np.asarray(col)) + y) / np.sqrt(d[rows])
    m = d.size
    return sp.csr_matrix((g, np.asarray(col), np.asarray(rowptr)), shape=(m, m))


def precond_loss_grad_f64(rowptr, col, val, B, p, X=None):
    """Loss and gradient with respect to the FP64 parameters p (no rounding).  With the paired
    solutions X the target of A G^T G b_c is A x_c, else b_c."""
    import scipy.sparse as sp
    p = np.asarray(p, np.float64)
    B = np.asarray(B, np.float64)
    m, ncols = B.shape
    feat, rows, d = precond_features(rowptr, col, val)
    F = feat.astype(np.float64)
    h1, h2, y = _mlp_forward(F, p)
    cols = np.asarray(col)
    sc = 1.0 / np.sqrt(d[rows])
    G = sp.csr_matrix((((rows == cols) + y) * sc, cols, np.asarray(rowptr)), shape=(m, m))
    A = sp.csr_matrix((np.asarray(val, np.float64), cols, np.asarray(rowptr)), shape=(m, m))
    bb = (B * B).sum(0)
    w = np.where(bb > 0, 1.0 / (ncols * np.where(bb > 0, bb, 1.0)), 0.0)
    Y = G @ B
    Z = G.T @ Y
    R = A @ Z - (B if X is None else A @ np.asarray(X, np.float64))
    loss = float((w * (R * R).sum(0)).sum())
    Phi = A @ (2.0 * w * R)          # d loss / d Z
    GPhi = G @ Phi                   # d loss / d Y
    dG = (Phi[cols] * Y[rows]).sum(1) + (GPhi[rows] * B[cols]).sum(1)
    return loss, _mlp_backward(F, h1, h2, dG * sc, p)


def precond_loss_grad(rowptr, col, val, B, params, X=None):
    """As the library defines it: parameters rounded to BF16 first."""
    return precond_loss_grad_f64(rowptr, col, val, B, bf16_round(params), X)
