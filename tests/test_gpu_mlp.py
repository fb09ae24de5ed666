"""The warm-start network's GPU kernels against the FP64 oracle, and what the trained network saves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import meshgen  # noqa: E402
import oracle  # noqa: E402
import paper_1705_10887_gb300 as sb  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sb.build()
    sb.library()


def test_gradient_matches_oracle():
    rng = np.random.default_rng(2)
    for N in (1, 127, 1000):
        X = rng.normal(size=(N, 6)).astype(np.float32)
        T = rng.normal(size=N).astype(np.float32)
        p = (rng.normal(size=sb.MLP_PARAMS) * 0.3).astype(np.float32)
        loss, g = sb.mlp_gradient(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(p).cuda())
        lo, go = oracle.mlp_loss_grad(X, T, p)
        g = g.cpu().numpy()
        # FP32 arithmetic against FP64 on the same BF16 weights
        assert abs(loss - lo) <= 1e-5 * max(lo, 1e-3)
        np.testing.assert_allclose(g, go, rtol=0, atol=2e-5 * np.abs(go).max())


def _torus_system(nu=120, nv=100, l=192, seed=5):
    import scipy.sparse as sp
    m = meshgen.torus(nu, nv, 1.0, 0.3, 0.2, seed=seed)
    g = oracle.mesh_operators(m.xyz, m.faces)
    n = g.n
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    A = sp.csr_matrix((g.A, (rows, g.col)), shape=(n, n))
    L = (sp.diags(np.asarray(A.sum(1)).ravel()) - A).tocsr()
    idx, _ = oracle.fps(g, l, 0)
    u = np.setdiff1d(np.arange(n), idx)
    Luu = L[u][:, u].tocsr()
    Luu.sort_indices()
    return m, g, idx, Luu, A[u][:, idx].toarray()


@pytest.mark.parametrize("ncols, dense, pairs", [(64, False, False), (40, True, False), (1, False, False),
                                                 (32, False, True)])
def test_precond_gradient_matches_oracle(ncols, dense, pairs):
    import scipy.sparse.linalg as sla
    rng = np.random.default_rng(ncols)
    _, _, _, Luu, Aub = _torus_system(60, 50, 48)
    B = rng.normal(size=(Luu.shape[0], ncols)) if dense else Aub[:, :ncols]
    X = sla.splu(Luu.tocsc()).solve(B) * (1 + 1e-3 * rng.normal(size=B.shape)) if pairs else None
    p = (rng.normal(size=sb.MLP_PARAMS) * 0.2).astype(np.float32)
    args = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (Luu.indptr.astype(np.int32),
                                                                        Luu.indices.astype(np.int32), Luu.data, B)]
    Xd = torch.from_numpy(X).cuda() if pairs else None
    loss, g = sb.precond_gradient(*args, torch.from_numpy(p).cuda(), Xd)
    lo, go = oracle.precond_loss_grad(Luu.indptr, Luu.indices, Luu.data, B, p, X)
    g = g.cpu().numpy()
    # FP32 sparse products and network against FP64 on the same BF16 weights
    assert abs(loss - lo) <= 2e-4 * lo
    np.testing.assert_allclose(g, go, rtol=0, atol=2e-3 * np.abs(go).max())
    # host arrays give the same result as device arrays
    loss_h, g_h = sb.precond_gradient(Luu.indptr.astype(np.int32), Luu.indices.astype(np.int32), Luu.data, B, p, X)
    assert abs(loss_h - lo) <= 2e-4 * lo


def test_precond_gradient_rejects_bad_input():
    _, _, _, Luu, Aub = _torus_system(30, 25, 12)
    p = np.zeros(sb.MLP_PARAMS, np.float32)
    rp, ci, v = Luu.indptr.astype(np.int32), Luu.indices.astype(np.int32), Luu.data.copy()
    with pytest.raises(sb.SbhaError):
        sb.precond_gradient(rp, ci, v, np.zeros((Luu.shape[0], 0)), p)
    v_bad = v.copy()
    v_bad[Luu.indptr[3] + np.flatnonzero(Luu.indices[Luu.indptr[3]:Luu.indptr[4]] == 3)[0]] = -1.0
    with pytest.raises(sb.SbhaError):
        sb.precond_gradient(rp, ci, v_bad, Aub[:, :4], p)
    ci_bad = ci.copy()
    ci_bad[0] = Luu.shape[0] + 5
    with pytest.raises(sb.SbhaError):
        sb.precond_gradient(rp, ci_bad, v, Aub[:, :4], p)


def test_learned_preconditioner_gain_and_parity():
    m, g, idx, _, _ = _torus_system()
    xyz, faces, didx = (torch.from_numpy(a).cuda() for a in (m.xyz, m.faces, idx))
    Pd = oracle.interpolation(oracle.biharmonic(g), idx)
    res = {}
    for pc in (sb.PRECOND_JACOBI, sb.PRECOND_MLP):
        o = sb.opts_default(precond=pc, precision=sb.PREC_FP32_REFINE, cg_rtol=1e-8)
        rowptr, col, val = sb.operator(xyz, faces, didx, 12, o)
        st = sb.last_stats()
        rp, cc, vv = rowptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
        rows = np.repeat(np.arange(m.n), np.diff(rp))
        res[pc] = (st, rp, cc, np.abs(vv - Pd[rows, cc]).max())
        assert st["cg_max_rel_residual"] <= 1e-8
    st_j, st_m = res[sb.PRECOND_JACOBI][0], res[sb.PRECOND_MLP][0]
    print("jacobi", {k: st_j[k] for k in ("cg_iterations", "e_iterations_jacobi", "k_iterations")})
    print("mlp", {k: st_m[k] for k in ("cg_iterations", "e_iterations_jacobi", "e_iterations_learned", "k_iterations",
                                      "mlp_loss_first",
                                      "mlp_loss_last", "mlp_train_entries", "mlp_ms_pilot", "mlp_ms_train")})
    assert st_m["mlp_trained"] == 1 and st_m["mlp_fallback"] == 0
    assert st_m["mlp_train_columns"] == 32 and st_m["mlp_train_entries"] > 0
    assert st_m["mlp_loss_last"] < 0.5 * st_m["mlp_loss_first"]
    # the learned preconditioner needs far fewer iterations than Jacobi on the same solves (whether a
    # correction of the biharmonic residual follows depends on rounding, so corrections are not compared)
    assert st_m["e_iterations_learned"] < 0.7 * st_j["e_iterations_jacobi"], (st_j, st_m)
    assert st_m["k_iterations"] < 0.7 * st_j["k_iterations"], (st_j, st_m)
    # same pattern and operator to the solver tolerance
    assert np.array_equal(res[sb.PRECOND_JACOBI][1], res[sb.PRECOND_MLP][1])
    assert res[sb.PRECOND_MLP][3] < 1e-6 and res[sb.PRECOND_JACOBI][3] < 1e-6
