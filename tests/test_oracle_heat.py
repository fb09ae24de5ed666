"""Pins of oracle.heat_geodesics (the heat method, Crane et al. 2013, which the paper's experiments use
for their distances) against exact distances on surfaces where they are known: the plane and the
sphere.  The method is approximate, with an error of the order of the mesh spacing h at t = h^2, so
the pins bound the error by a small multiple of h and check that it shrinks under refinement; a
sign slip, a transposed gradient or a dropped factor in the divergence fails them."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import meshgen  # noqa: E402
import oracle  # noqa: E402


def grid_error(k, jitter=0.0):
    h = 1.0 / (k - 1)
    m = meshgen.flat_grid(k, k, h, jitter=jitter, seed=1)
    c = (k // 2) * (k + 1)
    D = oracle.heat_geodesics(m.xyz, m.faces, [c, 0])
    E = np.linalg.norm(m.xyz - m.xyz[c], axis=1)
    E0 = np.linalg.norm(m.xyz - m.xyz[0], axis=1)
    assert D[0, c] == 0.0 and D[1, 0] == 0.0
    return h, np.abs(D[0] - E).max(), np.abs(D[1] - E0).max()


def test_plane_distances_within_two_spacings():
    h, e_center, e_corner = grid_error(41)
    assert e_center <= 1.5 * h and e_corner <= 2.0 * h
    h, e_center, _ = grid_error(41, jitter=0.2)
    assert e_center <= 1.5 * h


def test_plane_error_shrinks_under_refinement():
    # the largest error (along the grid's diagonal bias) shrinks more slowly than h, but it does shrink
    errs = [grid_error(k)[1] for k in (11, 21, 41, 81)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[3] < 0.6 * errs[1]


def test_sphere_great_circle_distances():
    s = meshgen.icosphere(4)  # unit sphere, 2562 vertices
    src = [0, 1000]
    D = oracle.heat_geodesics(s.xyz, s.faces, src)
    h = np.mean([np.linalg.norm(s.xyz[f[0]] - s.xyz[f[1]]) for f in s.faces])
    for k, v in enumerate(src):
        gc = np.arccos(np.clip(s.xyz @ s.xyz[v], -1.0, 1.0))
        assert np.abs(D[k] - gc).max() <= h
