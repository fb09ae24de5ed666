"""Failure detection, exercised from the host without faulting the GPU.

- A solve that reaches its iteration limit returns SBHA_ENOCONV and still writes its outputs
  (cg_max_iter = 1); so does the eigensolver (eig_max_iter = 1).
- A learned preconditioner that goes bad (its factor overwritten with NaN on the host through
  sbha_opts.fault_inject) stalls its first solve; Jacobi takes over, the stats say so, and the
  operator still matches the FP64 oracle.
- A bounded device wait that runs out (the wait limit set to zero through sbha_set_wait_limit)
  makes the tensor-core product return SBHA_ETIMEOUT; the kernel drains its own work, frees its
  tensor memory and returns, and the next call on the same context is correct.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import meshgen  # noqa: E402
import oracle  # noqa: E402
import paper_1705_10887_gb300 as sb  # noqa: E402
from tests._report import col_rel_err, report  # noqa: E402

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


@pytest.fixture(scope="module")
def torus():
    m = meshgen.torus(60, 40, 1.0, 0.3, 0.2, seed=1)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 45, 0)
    Pd = oracle.interpolation(oracle.biharmonic(g), idx)
    return m, idx, Pd


def _dense(rowptr, col, val, n, l):
    rp, c, v = (t.cpu().numpy() for t in (rowptr, col, val))
    P = np.zeros((n, l))
    mask = np.zeros((n, l), bool)
    rows = np.repeat(np.arange(n), np.diff(rp))
    P[rows, c] = v
    mask[rows, c] = True
    return P, mask


@pytest.mark.parametrize("solver", [sb.SOLVER_FACTORED, sb.SOLVER_DIRECT])
def test_iteration_limit_reports_noconv_and_writes_outputs(torus, solver):
    m, idx, _ = torus
    o = sb.opts_default(cg_max_iter=1, refine_max=1, solver=solver)
    with pytest.raises(sb.SbhaError) as e:
        sb.operator(cuda(m.xyz), cuda(m.faces), cuda(idx), 16, o)
    assert e.value.status == 3
    rowptr, col, val = sb.operator(cuda(m.xyz), cuda(m.faces), cuda(idx), 16, o, allow_noconv=True)
    rp = rowptr.cpu().numpy()
    assert rp[0] == 0 and int(rp[-1]) == idx.size + (m.n - idx.size) * 16
    assert np.all(np.diff(rp) >= 1)
    P, _ = _dense(rowptr, col, val, m.n, idx.size)
    assert np.array_equal(P[idx], np.eye(idx.size))  # landmark rows are exact whatever the solve did
    assert sb.last_stats()["cg_max_rel_residual"] > 1e-11


def test_eigensolver_limit_reports_noconv(torus):
    m, idx, Pd = torus
    S = oracle.sparsify_rows(Pd, idx, 16)
    W = oracle.landmark_block(oracle.mesh_operators(m.xyz, m.faces), idx)
    with pytest.raises(sb.SbhaError) as e:
        sb.mds(m.n, cuda(S.rowptr), cuda(S.col), cuda(S.val), cuda(W), 3, sb.opts_default(eig_max_iter=1))
    assert e.value.status == 3


def test_poisoned_network_falls_back_to_jacobi(torus):
    m, idx, Pd = torus
    o = sb.opts_default(precision=sb.PREC_FP32_REFINE, precond=sb.PRECOND_MLP, fault_inject=sb.FAULT_MLP_NAN)
    rowptr, col, val = sb.operator(cuda(m.xyz), cuda(m.faces), cuda(idx), 16, o)
    st = sb.last_stats()
    assert st["mlp_trained"] == 1 and st["mlp_fallback"] == 1
    assert st["cg_max_rel_residual"] <= 1e-11 * 1.0001
    P, mask = _dense(rowptr, col, val, m.n, idx.size)
    err = col_rel_err(P, Pd, mask)
    report("poisoned_network", max_rel=err, fallback=st["mlp_fallback"])
    assert err <= 1e-8
    # without the injected fault the network is kept
    sb.operator(cuda(m.xyz), cuda(m.faces), cuda(idx), 16, sb.opts_default(precision=sb.PREC_FP32_REFINE,
                                                                              precond=sb.PRECOND_MLP))
    st = sb.last_stats()
    assert st["mlp_trained"] == 1 and st["mlp_fallback"] == 0


def test_wait_timeout_returns_and_leaves_the_context_usable():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((200, 300))
    B = rng.standard_normal((300, 130))
    Ad, Bd = cuda(A), cuda(B)
    prev = sb.set_wait_limit(0)  # every bounded wait gives up at once
    try:
        with pytest.raises(sb.SbhaError) as e:
            sb.dgemm(Ad, Bd, sb.DENSE_TC)
        assert e.value.status == 6
    finally:
        sb.set_wait_limit(-1)
    assert prev > 0 and sb.set_wait_limit(-1) == prev  # the default was restored
    C = sb.dgemm(Ad, Bd, sb.DENSE_TC).cpu().numpy()
    assert np.abs(C - A @ B).max() <= 1e-12 * np.abs(A).max() * np.abs(B).max() * A.shape[1]
