"""GPU parity of the heat-method geodesics (Crane et al. 2013; the distances of the paper's experiments)
against oracle.heat_geodesics, which follows the same four steps with direct sparse solves.

Tolerance: the GPU solves the Poisson step by block-CG to cg_rtol, so phi carries an error of about
kappa(L) cg_rtol relative (kappa ~ n for these meshes); the heat step is summed to 1e-15 relative per
entry.  With cg_rtol = 1e-12 the distances agree within 1e-7 of the largest."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")

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


@pytest.mark.parametrize("name", ["sphere4", "torus60x40"])
@pytest.mark.parametrize("prec", [sb.PREC_FP64, sb.PREC_FP32_REFINE])
def test_heat_geodesics_match_the_oracle(name, prec):
    mesh = {"sphere4": meshgen.icosphere(4), "torus60x40": meshgen.torus(60, 40, 1.0, 0.3, 0.2, seed=1)}[name]
    src = np.array([0, mesh.n // 3, mesh.n - 1], np.int32)
    o = sb.opts_default(precision=prec, cg_rtol=1e-12)
    D = sb.heat_geodesics(cuda(mesh.xyz), cuda(mesh.faces), cuda(src), 1.0, o).cpu().numpy()
    Do = oracle.heat_geodesics(mesh.xyz, mesh.faces, src)
    assert np.abs(D - Do).max() <= 1e-7 * np.abs(Do).max()
    assert np.all(D[np.arange(3), src] == 0.0)
    st = sb.last_stats()
    assert st["heat_sweeps"] > 0 and st["cg_max_rel_residual"] <= 1e-12 * 1.0001


def test_many_sources_in_chunks_and_great_circles():
    s = meshgen.icosphere(3)  # 642 vertices: 642 sources are two chunks of columns
    src = np.arange(s.n, dtype=np.int32)
    D = sb.heat_geodesics(cuda(s.xyz), cuda(s.faces), cuda(src), 1.0, sb.opts_default(cg_rtol=1e-12)).cpu().numpy()
    pick = np.array([0, 17, 511, 512, 600, s.n - 1])
    Do = oracle.heat_geodesics(s.xyz, s.faces, pick)
    assert np.abs(D[pick] - Do).max() <= 1e-7 * np.abs(Do).max()
    gc = np.arccos(np.clip(s.xyz @ s.xyz.T, -1.0, 1.0))
    h = np.mean([np.linalg.norm(s.xyz[f[0]] - s.xyz[f[1]]) for f in s.faces])
    assert np.abs(D - gc).max() <= 1.5 * h
    # host buffers give the same distances
    Dh = sb.heat_geodesics(s.xyz, s.faces, pick, 1.0, sb.opts_default(cg_rtol=1e-12))
    assert np.abs(Dh - D[pick]).max() <= 1e-9 * np.abs(Do).max()


def test_bad_source():
    s = meshgen.icosphere(1)
    with pytest.raises(sb.SbhaError) as e:
        sb.heat_geodesics(s.xyz, s.faces, np.array([0, s.n], np.int32))
    assert e.value.status == 1
