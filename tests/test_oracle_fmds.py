"""Pins of oracle.fmds_interpolation, H = P (M_bb + mu I + M_bu P_u)^{-1} mu (Sec. 3.4.2)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import meshgen  # noqa: E402
import oracle  # noqa: E402


def test_path_by_hand():
    # path 0 - 1 - 2 (generic graph: M = L^2 = [[2,-3,1],[-3,6,-3],[1,-3,2]]), landmarks 0 and 2:
    #   P_u = -M_uu^{-1} M_ub = [1/2, 1/2];  M_bu P_u = [[-3/2,-3/2],[-3/2,-3/2]];
    #   S = M_bb + mu I + M_bu P_u = [[1/2 + mu, -1/2], [-1/2, 1/2 + mu]], eigenvalues mu (along [1,1])
    #   and mu + 1 (along [1,-1]); at mu = 1, mu S^{-1} = [[3/4, 1/4], [1/4, 3/4]], so
    #   H = P mu S^{-1} = [[3/4, 1/4], [1/2, 1/2], [1/4, 3/4]].
    g = oracle.graph_operators(np.array([0, 1, 3, 4], np.int32), np.array([1, 0, 2, 1], np.int32))
    M = oracle.biharmonic(g)
    idx = np.array([0, 2], np.int32)
    P = oracle.interpolation(M, idx)
    np.testing.assert_allclose(P, [[1.0, 0.0], [0.5, 0.5], [0.0, 1.0]], atol=1e-15)
    H = oracle.fmds_interpolation(M, idx, P, 1.0)
    np.testing.assert_allclose(H, [[0.75, 0.25], [0.5, 0.5], [0.25, 0.75]], atol=1e-14)


def test_rows_sum_to_one_and_large_mu_gives_p():
    # P_u 1 = 1 and M 1 = 0 give S 1 = mu 1, so H 1 = P 1 = 1; as mu grows, mu S^{-1} -> I and H -> P
    m = meshgen.torus(16, 12, 1.0, 0.3, 0.2, seed=4)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 20, 0)
    M = oracle.biharmonic(g)
    P = oracle.interpolation(M, idx)
    H = oracle.fmds_interpolation(M, idx, P, 50.0)
    assert np.abs(H.sum(axis=1) - 1.0).max() < 1e-10
    assert np.abs(H[idx] - np.eye(20)).max() > 1e-6  # landmark values are no longer interpolated exactly
    assert np.abs(oracle.fmds_interpolation(M, idx, P, 1e12) - P).max() < 1e-8
