"""The synthetic inputs have the sizes and shapes the workloads state, and the benchmark's sampled
stress is the oracle's stress when the sample is every vertex."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import meshgen  # noqa: E402
import oracle  # noqa: E402


def _edges_used_once(faces):
    e = np.sort(np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]]), axis=1)
    _, counts = np.unique(e, axis=0, return_counts=True)
    return int(np.sum(counts == 1))


def test_workload_sizes():
    m, w = meshgen.workload("icosphere3_l32")
    assert (m.n, len(m.faces), w["l"], w["p_row"], w["k"]) == (642, 1280, 32, 8, 3)
    assert _edges_used_once(m.faces) == 0  # closed
    m, w = meshgen.workload("torus250x200_l500")
    assert (m.n, len(m.faces), w["l"], w["p_row"]) == (50000, 100000, 500, 16)
    assert _edges_used_once(m.faces) == 0  # closed
    m, w = meshgen.workload("patch448_l2000")
    assert (m.n, w["l"], w["p_row"]) == (448 * 448, 2000, 16)
    assert _edges_used_once(m.faces) > 0  # an open patch


def test_batch_sizes_are_log_uniform_and_in_range():
    meshes = meshgen.mesh_batch(64, 5000, 100000, seed=1)
    n = np.array([m.n for m in meshes])
    assert len(meshes) == 64 and n.min() >= 4000 and n.max() <= 110000
    # log-uniform: about half the meshes below the geometric mean of the range
    below = np.sum(n < np.sqrt(5000 * 100000))
    assert 20 <= below <= 44


def test_bench_sampled_stress_is_the_oracle_stress_on_every_vertex():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    rng = np.random.default_rng(0)
    pts = rng.random((60, 3))
    E = np.sum((pts[:, None, :] - pts[None, :, :]) ** 2, axis=2)
    Z = pts[:, :2] + 0.01 * rng.normal(size=(60, 2))
    a = bench.normalised_stress(Z, E, np.arange(60))
    b = oracle.stress(Z, E)
    assert abs(a - b) <= 1e-12 * b
