"""GPU parity of sbha_bha_error, the sampled relative error of K~ = P W P^T (Sec. 4.1), against
oracle.bha_error on the same operator, landmark block and exact distance rows."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import meshgen  # noqa: E402
import oracle  # noqa: E402
import paper_1705_10887_gb300 as sb  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sb.build()
    sb.library()


def case(mesh, l, p):
    g = oracle.mesh_operators(mesh.xyz, mesh.faces)
    idx, _ = oracle.fps(g, l, 0)
    P = oracle.sparsify_rows(oracle.interpolation(oracle.biharmonic(g), idx), idx, p)
    return g, idx, P, oracle.landmark_block(g, idx)


def gpu_err(P, W, rows, K, squared):
    return sb.bha_error(cuda(P.rowptr), cuda(P.col), cuda(P.val), cuda(W), cuda(rows.astype(np.int32)), cuda(K),
                        squared)


@pytest.mark.parametrize("squared", [False, True])
@pytest.mark.parametrize("name", ["icosphere3", "torus60x40"])
def test_small_meshes_every_row_and_a_sample(name, squared):
    mesh, l, p = {"icosphere3": (meshgen.icosphere(3, noise=0.01, seed=0), 32, 8),
                  "torus60x40": (meshgen.torus(60, 40, 1.0, 0.3, 0.2, seed=1), 45, 16)}[name]
    g, idx, P, W = case(mesh, l, p)
    K = oracle.geodesics(g, np.arange(mesh.n, dtype=np.int32))
    for rows in (np.arange(mesh.n), np.sort(np.random.default_rng(2).choice(mesh.n, 77, replace=False))):
        num, den = gpu_err(P, W, rows, K[rows], squared)
        on, od = oracle.bha_error(P, W, rows, K[rows], squared)
        assert abs(num - on) <= 1e-10 * on and abs(den - od) <= 1e-12 * od
    assert 0.0 < num / den < 0.1


def test_host_buffers_empty_sample_and_errors():
    mesh = meshgen.icosphere(2, noise=0.01, seed=1)
    g, idx, P, W = case(mesh, 20, 6)
    rows = np.array([0, 3, 100], np.int32)
    K = oracle.geodesics(g, rows)
    h = sb.bha_error(P.rowptr, P.col, P.val, W, rows, K)
    d = gpu_err(P, W, rows, K, False)
    assert abs(h[0] - d[0]) <= 1e-13 * d[0] and h[1] == d[1]
    assert sb.bha_error(P.rowptr, P.col, P.val, W, np.zeros(0, np.int32), np.zeros((0, mesh.n))) == (0.0, 0.0)
    with pytest.raises(sb.SbhaError) as e:  # a sampled row outside [0, n)
        sb.bha_error(P.rowptr, P.col, P.val, W, np.array([mesh.n], np.int32), np.zeros((1, mesh.n)))
    assert e.value.status == 1
    bad = P.col.copy()
    bad[5] = 20  # a column outside [0, l)
    with pytest.raises(sb.SbhaError) as e:
        sb.bha_error(P.rowptr, bad, P.val, W, rows, K)
    assert e.value.status == 1


def test_torus250x200_l500_sampled_rows():
    """The benchmark mesh and operator: 300 sampled rows of exact distances from the GPU."""
    mesh, w = meshgen.workload("torus250x200_l500")
    l, p = w["l"], w["p_row"]
    x, f = cuda(mesh.xyz), cuda(mesh.faces)
    idx = sb.landmarks(x, f, l, 0)
    rowptr, col, val = sb.operator(x, f, idx, p)
    W = sb.landmark_distances(x, f, idx)
    rows = np.sort(np.random.default_rng(3).choice(mesh.n, 300, replace=False)).astype(np.int32)
    K = sb.geodesics(x, f, cuda(rows))
    P = oracle.CSR(rowptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy(), l)
    Wh, Kh = W.cpu().numpy(), K.cpu().numpy()
    for squared in (False, True):
        num, den = sb.bha_error(rowptr, col, val, W, cuda(rows), K, squared)
        on, od = oracle.bha_error(P, Wh, rows, Kh, squared)
        assert abs(num - on) <= 1e-10 * on and abs(den - od) <= 1e-12 * od
