"""Pins for the oracle's cotangent adjacency, lumped mass and biharmonic operator (Sec. 2.2)."""
import math

import numpy as np
import pytest

import meshgen
import oracle
from tests import _brute


def equilateral_lattice(nu, nv):
    """Flat triangular lattice with unit edges: p(i, j) = i (1, 0) + j (-1/2, sqrt(3)/2)."""
    m = meshgen.flat_grid(nu, nv)
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    m.xyz[:, 0] = (i - 0.5 * j).ravel()
    m.xyz[:, 1] = (j * math.sqrt(3.0) / 2.0).ravel()
    return m


def interior_mask(m, rings=1):
    """Vertices at least ``rings`` edge steps from the boundary of an open grid mesh."""
    edges = _brute.edge_list(m.faces)
    # boundary edges belong to exactly one face
    e = np.concatenate([m.faces[:, [0, 1]], m.faces[:, [1, 2]], m.faces[:, [2, 0]]]).astype(np.int64)
    e.sort(axis=1)
    uniq, cnt = np.unique(e, axis=0, return_counts=True)
    bnd = np.zeros(m.n, bool)
    bnd[uniq[cnt == 1].ravel()] = True
    adj = [[] for _ in range(m.n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    far = ~bnd
    for _ in range(rings - 1):
        far = far & np.array([all(far[w] for w in adj[v]) for v in range(m.n)])
    return far


def test_lumped_mass_sums_to_area():
    for m in (meshgen.icosphere(2, noise=0.01, seed=1), meshgen.torus(20, 15, seed=2), meshgen.sphere_patch_bumps(30)):
        g = oracle.mesh_operators(m.xyz, m.faces)
        area = _brute.triangle_areas(m.xyz, m.faces)
        assert abs(g.D.sum() - area.sum()) <= 1e-13 * area.sum()
        Dref = np.zeros(m.n)
        for k in range(3):
            np.add.at(Dref, m.faces[:, k], area / 3.0)
        np.testing.assert_allclose(g.D, Dref, rtol=1e-14)


def test_icosphere_area_tends_to_4pi():
    errs = []
    for level in (2, 3, 4):
        m = meshgen.icosphere(level)
        g = oracle.mesh_operators(m.xyz, m.faces)
        errs.append(abs(g.D.sum() - 4 * math.pi))
    # inscribed polyhedra converge to the sphere's area at second order: the error quarters per level
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5 and errs[2] < 0.02


def test_equilateral_lattice_cotangent_closed_form():
    m = equilateral_lattice(8, 7)
    g = oracle.mesh_operators(m.xyz, m.faces)
    inner = interior_mask(m)
    for i in range(m.n):
        for e in range(g.rowptr[i], g.rowptr[i + 1]):
            j = g.col[e]
            if inner[i] and inner[j]:
                assert abs(g.A[e] - 1.0 / math.sqrt(3.0)) < 1e-14
        if inner[i]:
            assert abs(g.D[i] - math.sqrt(3.0) / 2.0) < 1e-14


def test_weight_sums():
    # equilateral lattice: an interior vertex has six unit edges of weight 1/sqrt(3), so V = 2 sqrt(3)
    m = equilateral_lattice(8, 7)
    g = oracle.mesh_operators(m.xyz, m.faces)
    V = oracle.weight_sums(g)
    inner = interior_mask(m)
    assert np.abs(V[inner] - 2.0 * math.sqrt(3.0)).max() < 1e-14
    # every row: the exactly rounded sum of its weights, up to the rounding of a short left fold
    for m in (meshgen.torus(20, 15, seed=3), meshgen.sphere_patch_bumps(20, 4, seed=2)):
        g = oracle.mesh_operators(m.xyz, m.faces)
        V = oracle.weight_sums(g)
        for i in range(m.n):
            row = g.A[g.rowptr[i]:g.rowptr[i + 1]]
            exact = math.fsum(row)
            assert abs(V[i] - exact) <= 8 * np.finfo(float).eps * np.abs(row).sum()
        # the constant function is in the kernel of L = V - A
        L = _brute.dense_laplacian(g)
        assert np.abs(np.diag(L) - V).max() <= 1e-14 * np.abs(V).max()


def test_cotangent_weights_symmetric_bitwise():
    m = meshgen.torus(20, 15, seed=3)
    g = oracle.mesh_operators(m.xyz, m.faces)
    lookup = {}
    for i in range(m.n):
        for e in range(g.rowptr[i], g.rowptr[i + 1]):
            lookup[(i, int(g.col[e]))] = g.A[e]
    for (i, j), a in lookup.items():
        assert lookup[(j, i)] == a


def test_laplacian_annihilates_linear_functions_on_planar_mesh():
    m = meshgen.flat_grid(12, 10, jitter=0.15, seed=4)
    g = oracle.mesh_operators(m.xyz, m.faces)
    L = _brute.dense_laplacian(g)
    inner = interior_mask(m)
    for f in (m.xyz[:, 0], m.xyz[:, 1], 2.0 * m.xyz[:, 0] - 3.0 * m.xyz[:, 1] + 0.5):
        r = L @ f
        assert np.abs(r[inner]).max() < 1e-12
        assert np.abs(r[~inner]).max() > 1e-3  # the boundary really is different


@pytest.fixture(scope="module")
def operator_cases():
    out = []
    for m in (meshgen.icosphere(2, noise=0.01, seed=1), meshgen.torus(16, 12, seed=2),
              meshgen.flat_grid(12, 10, jitter=0.15, seed=4), meshgen.sphere_patch_bumps(14)):
        g = oracle.mesh_operators(m.xyz, m.faces)
        out.append((m, g, oracle.biharmonic(g)))
    return out


def test_biharmonic_symmetric_constant_nullspace_psd(operator_cases):
    for m, g, M in operator_cases:
        Md = M.todense()
        assert np.array_equal(Md, Md.T), "M must be bitwise symmetric"
        scale = np.abs(Md).max()
        assert np.abs(Md @ np.ones(m.n)).max() < 1e-12 * scale
        w = np.linalg.eigvalsh(Md)
        assert w.min() > -1e-12 * w.max()
        # exactly one zero eigenvalue per connected component (here: one)
        assert np.sum(np.abs(w) < 1e-10 * w.max()) == 1


def test_biharmonic_pattern_is_two_ring(operator_cases):
    for m, g, M in operator_cases:
        A = np.zeros((m.n, m.n), bool)
        for a, b in _brute.edge_list(m.faces):
            A[a, b] = A[b, a] = True
        one = A | np.eye(m.n, dtype=bool)
        two = (one.astype(np.int64) @ one.astype(np.int64)) > 0
        pat = np.zeros((m.n, m.n), bool)
        for i in range(m.n):
            pat[i, M.col[M.rowptr[i] : M.rowptr[i + 1]]] = True
        assert np.array_equal(pat, two)


def test_biharmonic_equals_dense_triple_product(operator_cases):
    for m, g, M in operator_cases:
        L = _brute.dense_laplacian(g)
        ref = L.T @ np.diag(1.0 / g.D) @ L
        np.testing.assert_allclose(M.todense(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_biharmonic_annihilates_linear_functions_away_from_boundary():
    m = meshgen.flat_grid(14, 12, jitter=0.15, seed=7)
    g = oracle.mesh_operators(m.xyz, m.faces)
    M = oracle.biharmonic(g).todense()
    inner2 = interior_mask(m, rings=2)
    for f in (m.xyz[:, 0], m.xyz[:, 1]):
        r = M @ f
        assert np.abs(r[inner2]).max() < 1e-11 * np.abs(M).max()


def test_invalid_faces_rejected():
    m = meshgen.icosphere(1)
    bad = m.faces.copy()
    bad[0, 0] = m.n  # out of range
    with pytest.raises(oracle.OracleError):
        oracle.mesh_operators(m.xyz, bad)
    bad = m.faces.copy()
    bad[0, 1] = bad[0, 0]  # repeated vertex
    with pytest.raises(oracle.OracleError):
        oracle.mesh_operators(m.xyz, bad)
    # an edge shared by three faces
    tri = np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]], np.int32)
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1]], float)
    with pytest.raises(oracle.OracleError):
        oracle.mesh_operators(xyz, tri)
