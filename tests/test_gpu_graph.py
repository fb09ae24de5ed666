"""GPU parity on generic graphs (Sec. 2.2: D = I, A = the 0/1 adjacency, geodesics along the
graph's edges) against the oracle run on the same graph."""
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
RTOL = 1e-11


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sb.build()
    sb.library()


_cache = {}


def knn_case():
    if "knn" not in _cache:
        rp, col, length, _ = meshgen.knn_graph(3000, 6, seed=1)
        l, p = 40, 12
        g = oracle.graph_operators(rp, col, length)
        idx, _ = oracle.fps(g, l, 0)
        W = oracle.landmark_block(g, idx)
        M = oracle.biharmonic(g)
        Pd = oracle.interpolation(M, idx)
        S = oracle.sparsify_rows(Pd, idx, p)
        Z, theta = oracle.mds_gram(S, W, 3)
        Md = M.todense()
        unk = np.setdiff1d(np.arange(rp.size - 1), idx)
        lam = np.linalg.eigvalsh(Md[np.ix_(unk, unk)])[0]
        bound = RTOL * np.linalg.norm(Md[np.ix_(unk, idx)], axis=0) / lam + 1e-12
        _cache["knn"] = dict(rp=rp, col=col, length=length, l=l, p=p, idx=idx, Pd=Pd, S=S, Z=Z, theta=theta,
                             bound=bound)
    return _cache["knn"]


@pytest.mark.parametrize("prec,precond", [(sb.PREC_FP64, sb.PRECOND_JACOBI), (sb.PREC_FP32_REFINE, sb.PRECOND_MLP)])
def test_knn_graph_operator_and_embedding(prec, precond):
    r = knn_case()
    n, l, p = r["rp"].size - 1, r["l"], r["p"]
    o = sb.opts_default(precision=prec, precond=precond, cg_rtol=RTOL)
    Z, ev, idx = sb.graph_embed(cuda(r["rp"]), cuda(r["col"]), l, p, 3, 0, cuda(r["length"]), o)
    assert np.array_equal(idx.cpu().numpy(), r["idx"])
    rowptr, col, val = sb.graph_operator(cuda(r["rp"]), cuda(r["col"]), idx, p, cuda(r["length"]), o)
    assert sb.last_stats()["cg_max_rel_residual"] <= RTOL * 1.0001
    rp, c, v = rowptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    P = np.zeros((n, l))
    mask = np.zeros((n, l), bool)
    P[rows, c] = v
    mask[rows, c] = True
    assert np.array_equal(P[r["idx"]], np.eye(l))
    assert not ((np.abs(P - r["Pd"]) * mask) > r["bound"][None, :]).any()
    Smask = np.zeros_like(mask)
    Smask[np.repeat(np.arange(n), np.diff(r["S"].rowptr)), r["S"].col] = True
    for i in np.nonzero(np.any(mask != Smask, axis=1))[0]:
        a = np.sort(np.abs(r["Pd"][i]))[::-1]
        assert a[p - 1] - a[p] <= 2 * r["bound"].max()
    np.testing.assert_allclose(ev.cpu().numpy(), r["theta"], rtol=1e-8)
    Z = Z.cpu().numpy()
    G1, G2 = Z @ Z.T, r["Z"] @ r["Z"].T
    assert np.abs(G1 - G2).max() <= 1e-6 * np.abs(G2).max()


def test_grid_graph_hop_landmarks_bit_exact():
    """Integer hop distances make farthest-point ties everywhere: the lowest vertex wins on both sides."""
    rp, col = meshgen.grid_graph(60, 45)
    g = oracle.graph_operators(rp, col)
    idx_o, _ = oracle.fps(g, 50, 0)
    _, _, idx = sb.graph_embed(cuda(rp), cuda(col), 50, 8, 3, 0)
    assert np.array_equal(idx.cpu().numpy(), idx_o)


def test_host_graph_and_malformed_graphs():
    r = knn_case()
    _, evh, idxh = sb.graph_embed(r["rp"], r["col"], r["l"], r["p"], 3, 0, r["length"])
    assert isinstance(evh, np.ndarray) and np.array_equal(idxh, r["idx"])
    rp, col = meshgen.grid_graph(6, 5)
    idx = np.array([0, 29], np.int32)

    def expect_einval(rp_, col_, length=None):
        with pytest.raises(sb.SbhaError) as e:
            sb.graph_operator(rp_, col_, idx, 2, length)
        assert e.value.status == 1

    bad = col.copy()
    bad[0] = 0  # a self loop at vertex 0
    expect_einval(rp, bad)
    bad = col.copy()
    bad[0], bad[1] = bad[1], bad[0]  # row 0 not ascending
    expect_einval(rp, bad)
    bad = col.copy()
    bad[1] = 7  # 0 - 7 without its reverse edge
    expect_einval(rp, bad)
    length = np.ones(col.size)
    length[0] = 2.0  # the reverse edge has another length
    expect_einval(rp, col, length)
    length = np.ones(col.size)
    length[3] = -1.0
    expect_einval(rp, col, length)
