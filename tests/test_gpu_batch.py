"""A batch of uneven meshes through one call: every mesh against the FP64 oracle run end to end (landmarks
bit for bit, eigenvalues and Z Z^T at the mixed-precision bars), and against the single-mesh pipeline."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import meshgen  # noqa: E402
import oracle  # noqa: E402
import paper_1705_10887_gb300 as sb  # noqa: E402
from tests._report import gram_rel_err, report  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sb.build()
    sb.library()


def _meshes():
    ms = [meshgen.torus(60, 51, 1.0, 0.3, 0.2, seed=3), meshgen.icosphere(3, 0.01, 0), meshgen.torus(40, 30, 1.0, 0.3, 0.2, seed=4),
          meshgen.icosphere(2, 0.01, 1), meshgen.torus(90, 70, 1.0, 0.3, 0.2, seed=5)]
    ls = [max(8, m.n // 40) for m in ms]
    return ms, ls


@pytest.mark.parametrize("workers, precond", [(0, sb.PRECOND_JACOBI), (1, sb.PRECOND_JACOBI), (3, sb.PRECOND_MLP)])
def test_batch_equals_single(workers, precond):
    ms, ls = _meshes()
    firsts = [i % 3 for i in range(len(ms))]
    o = sb.opts_default(precision=sb.PREC_FP32_REFINE, precond=precond, cg_rtol=1e-10)
    dev = [(torch.from_numpy(m.xyz).cuda(), torch.from_numpy(m.faces).cuda()) for m in ms]
    out = sb.embed_batch(dev, ls, 8, 3, firsts, o, workers=workers)
    st = sb.last_stats()
    assert st["cg_max_rel_residual"] <= 1e-10
    for (x, f), l, fi, (Z, ev, idx) in zip(dev, ls, firsts, out):
        Z1, ev1, idx1 = sb.embed(x, f, l, 8, 3, fi, o)
        assert torch.equal(idx.cpu(), idx1.cpu())
        np.testing.assert_allclose(ev.cpu().numpy(), ev1.cpu().numpy(), rtol=1e-8)
        G, G1 = (Z @ Z.T).cpu().numpy(), (Z1 @ Z1.T).cpu().numpy()
        assert np.abs(G - G1).max() <= 1e-6 * np.abs(G1).max()


def test_batch_host_arrays_and_errors():
    ms, ls = _meshes()
    out = sb.embed_batch([(m.xyz, m.faces) for m in ms[:2]], ls[:2], 8, 3)
    assert isinstance(out[0][0], np.ndarray) and out[1][0].shape == (ms[1].n, 3)
    bad = list(ls[:2])
    bad[1] = ms[1].n + 1
    with pytest.raises(sb.SbhaError) as e:
        sb.embed_batch([(m.xyz, m.faces) for m in ms[:2]], bad, 8, 3)
    assert "mesh 1" in str(e.value)


def test_every_mesh_of_a_batch_against_the_oracle():
    """Eight meshes of uneven size (1,000-8,000 vertices, log-uniform, seed 4; spheres and tori), l = 2% of
    each, learned + mixed precision, one call: each mesh's landmarks bit for bit, eigenvalues within 1e-8 and
    Z Z^T within 1e-6 of the oracle's end-to-end run on that mesh alone."""
    ms = meshgen.mesh_batch(8, 1000, 8000, seed=4)
    ls = [max(34, int(round(0.02 * m.n))) for m in ms]
    o = sb.opts_default(precision=sb.PREC_FP32_REFINE, precond=sb.PRECOND_MLP)
    dev = [(torch.from_numpy(m.xyz).cuda(), torch.from_numpy(m.faces).cuda()) for m in ms]
    out = sb.embed_batch(dev, ls, 12, 3, None, o, workers=4)
    worst_ev = worst_z = 0.0
    for m, l, (Z, ev, idx) in zip(ms, ls, out):
        ro = oracle.sbmds(m.xyz, m.faces, l, 12, 3, 0)
        assert np.array_equal(idx.cpu().numpy(), ro.idx)
        ev_err = float(np.max(np.abs(ev.cpu().numpy() - ro.theta) / np.abs(ro.theta)))
        z_err = gram_rel_err(Z.cpu().numpy(), ro.Z)
        worst_ev, worst_z = max(worst_ev, ev_err), max(worst_z, z_err)
        assert ev_err <= 1e-8 and z_err <= 1e-6, f"mesh n={m.n}: {ev_err:.2e} {z_err:.2e}"
    report("batch_vs_oracle", meshes=len(ms), eval_rel=worst_ev, zzt_rel=worst_z)
