"""GPU parity of the FMDS interpolation matrix H = P (M_bb + mu I + M_bu P_u)^{-1} mu (Sec. 3.4.2)
against oracle.fmds_interpolation on the oracle's dense operator.  The GPU's P carries the solve's
error (cg_rtol 1e-11); the l x l system is well conditioned at mu = 50, so H agrees to ~1e-9."""
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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sb.build()
    sb.library()


@pytest.mark.parametrize("name,l", [("icosphere3", 32), ("torus60x40", 45)])
@pytest.mark.parametrize("dense", [sb.DENSE_TC, sb.DENSE_FP64])
def test_fmds_matches_the_oracle(name, l, dense):
    mesh = {"icosphere3": meshgen.icosphere(3, noise=0.01, seed=0),
            "torus60x40": meshgen.torus(60, 40, 1.0, 0.3, 0.2, seed=1)}[name]
    g = oracle.mesh_operators(mesh.xyz, mesh.faces)
    idx, _ = oracle.fps(g, l, 0)
    M = oracle.biharmonic(g)
    Ho = oracle.fmds_interpolation(M, idx, oracle.interpolation(M, idx), 50.0)
    o = sb.opts_default(dense_mode=dense, precision=sb.PREC_FP32_REFINE)
    H = sb.fmds_operator(cuda(mesh.xyz), cuda(mesh.faces), cuda(idx), 50.0, o).cpu().numpy()
    assert np.abs(H - Ho).max() <= 1e-8 * np.abs(Ho).max()
    assert np.abs(H.sum(axis=1) - 1.0).max() <= 1e-8


def test_fmds_host_buffers_and_bad_mu():
    mesh = meshgen.icosphere(2, noise=0.01, seed=2)
    g = oracle.mesh_operators(mesh.xyz, mesh.faces)
    idx, _ = oracle.fps(g, 12, 0)
    Hh = sb.fmds_operator(mesh.xyz, mesh.faces, idx, 50.0)
    Hd = sb.fmds_operator(cuda(mesh.xyz), cuda(mesh.faces), cuda(idx), 50.0).cpu().numpy()
    assert isinstance(Hh, np.ndarray) and np.abs(Hh - Hd).max() <= 1e-12
    for mu in (0.0, -1.0, float("inf")):
        with pytest.raises(sb.SbhaError) as e:
            sb.fmds_operator(mesh.xyz, mesh.faces, idx, mu)
        assert e.value.status == 1
