"""GPU parity of the sBMDS eigen route (Sec. 3.3): thick-restart Lanczos on the n x n operator
-1/2 J P (W.W) P^T J, applied only through products with P, P^T and W.W.

The same eigenpairs have two independent oracle forms: the landmark-space Gram route
(oracle.mds_gram) and, for small n, the dense n x n matrix itself (oracle.mds_full of
E = P (W.W) P^T, which forms -1/2 J E J and diagonalises it by Jacobi)."""
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

CASES = {
    "icosphere3": (meshgen.icosphere(3, noise=0.01, seed=0), 32, 8),
    "torus60x40": (meshgen.torus(60, 40, 1.0, 0.3, 0.2, seed=1), 45, 16),
    "patch40": (meshgen.sphere_patch_bumps(40, 5, seed=2), 70, 12),
    "torus48x40_l600": (meshgen.torus(48, 40, 1.0, 0.3, 0.2, seed=3), 600, 10),
}


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sb.build()
    sb.library()


_cache = {}


def ref(name):
    if name not in _cache:
        m, l, p = CASES[name]
        g = oracle.mesh_operators(m.xyz, m.faces)
        idx, _ = oracle.fps(g, l, 0)
        W = oracle.landmark_block(g, idx)
        Pd = oracle.interpolation(oracle.biharmonic(g), idx)
        S = oracle.sparsify_rows(Pd, idx, p)
        _cache[name] = dict(mesh=m, l=l, p=p, W=W, S=S)
    return _cache[name]


def lanczos(r, k, **kw):
    o = sb.opts_default(eig_route=sb.EIG_LANCZOS, **kw)
    S = r["S"]
    Z, ev = sb.mds(r["mesh"].n, cuda(S.rowptr), cuda(S.col), cuda(S.val), cuda(r["W"]), k, o)
    return Z.cpu().numpy(), ev.cpu().numpy(), sb.last_stats()


def dense_P(S, n, l):
    P = np.zeros((n, l))
    for i in range(n):
        P[i, S.col[S.rowptr[i]:S.rowptr[i + 1]]] = S.val[S.rowptr[i]:S.rowptr[i + 1]]
    return P


@pytest.mark.parametrize("name", list(CASES))
def test_lanczos_matches_gram_route(name):
    r = ref(name)
    Zo, tho = oracle.mds_gram(r["S"], r["W"], 3)
    Z, ev, st = lanczos(r, 3)
    np.testing.assert_allclose(ev, tho, rtol=1e-8)
    G1, G2 = Z @ Z.T, Zo @ Zo.T
    assert np.abs(G1 - G2).max() <= 1e-6 * np.abs(G2).max()
    for q in range(3):  # the sign rule of the landmark route holds here too
        i = int(np.argmax(np.abs(Z[:, q])))
        assert Z[i, q] > 0
    assert st["eig_residual"] <= 1e3 * 1e-13
    assert st["eig_iterations"] >= 1


def test_lanczos_matches_dense_operator():
    """The n x n operator written out: -1/2 J P (W.W) P^T J, dense Jacobi eigenpairs."""
    r = ref("icosphere3")
    n, l = r["mesh"].n, r["l"]
    P = dense_P(r["S"], n, l)
    E = P @ (r["W"] * r["W"]) @ P.T
    Zo, tho = oracle.mds_full(E, 3)
    Z, ev, _ = lanczos(r, 3)
    np.testing.assert_allclose(ev, tho, rtol=1e-8)
    G1, G2 = Z @ Z.T, Zo @ Zo.T
    assert np.abs(G1 - G2).max() <= 1e-6 * np.abs(G2).max()


@pytest.mark.parametrize("name,k", [("patch40", 12), ("patch40", 20), ("torus48x40_l600", 12)])
def test_lanczos_thick_restarts(name, k):
    """More wanted pairs than the basis holds room for between restarts: the top-k values still
    match, and the run took more operator products than one basis fill (32)."""
    r = ref(name)
    _, tho = oracle.mds_gram(r["S"], r["W"], k)
    _, ev, st = lanczos(r, k)
    np.testing.assert_allclose(ev, tho, rtol=1e-8)
    assert st["eig_iterations"] > 32


def test_lanczos_end_to_end_embed():
    r = ref("torus60x40")
    m = r["mesh"]
    ro = oracle.sbmds(m.xyz, m.faces, r["l"], r["p"], 3, 0)
    o = sb.opts_default(eig_route=sb.EIG_LANCZOS, precision=sb.PREC_FP32_REFINE)
    Z, ev, idx = sb.embed(cuda(m.xyz), cuda(m.faces), r["l"], r["p"], 3, 0, o)
    assert np.array_equal(idx.cpu().numpy(), ro.idx)
    np.testing.assert_allclose(ev.cpu().numpy(), ro.theta, rtol=1e-8)
    Z = Z.cpu().numpy()
    G1, G2 = Z @ Z.T, ro.Z @ ro.Z.T
    assert np.abs(G1 - G2).max() <= 1e-6 * np.abs(G2).max()


def test_lanczos_host_buffers_and_batch():
    r = ref("patch40")
    S = r["S"]
    o = sb.opts_default(eig_route=sb.EIG_LANCZOS)
    Zh, evh = sb.mds(r["mesh"].n, S.rowptr, S.col, S.val, r["W"], 3, o)
    _, evd, _ = lanczos(r, 3)
    assert isinstance(Zh, np.ndarray)
    np.testing.assert_allclose(evh, evd, rtol=1e-12)
    a, b = CASES["icosphere3"][0], CASES["patch40"][0]
    out = sb.embed_batch([(cuda(a.xyz), cuda(a.faces)), (cuda(b.xyz), cuda(b.faces))], [32, 70], 8, 3, None, o)
    for (Zb, evb, _), mesh, l in zip(out, (a, b), (32, 70)):
        ro = oracle.sbmds(mesh.xyz, mesh.faces, l, 8, 3, 0)
        np.testing.assert_allclose(evb.cpu().numpy(), ro.theta, rtol=1e-8)


def test_lanczos_errors():
    r = ref("icosphere3")
    S = r["S"]
    with pytest.raises(sb.SbhaError) as e:  # k > min(n, 32) - 10
        lanczos(r, 23)
    assert e.value.status == 1
    with pytest.raises(sb.SbhaError) as e:
        sb.mds(r["mesh"].n, cuda(S.rowptr), cuda(S.col), cuda(S.val), cuda(r["W"]), 3, sb.opts_default(eig_route=7))
    assert e.value.status == 1
