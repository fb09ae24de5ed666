"""sbha_mds_static, the allocation-free variant of the scaling step, against sbha_mds and
against the FP64 oracle's scaling of the same operator.

Some callers cannot allocate device memory while they run the scaling step (they
reserve all device memory up front, or run in a loop where an allocation could stall
or fail).  sbha_mds_static serves them from a fixed workspace inside the library.
This file runs last (its name sorts last) so that a failing run of the whole suite has
already exercised everything else; it also passes when run alone in a new process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import meshgen  # noqa: E402
import oracle  # noqa: E402
import paper_1705_10887_gb300 as sb  # noqa: E402

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sb.build()
    lib = sb.library()
    m = meshgen.torus(40, 30, 1.0, 0.3, 0.2, seed=4)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 60, 0)
    W = oracle.landmark_block(g, idx)
    P = oracle.sparsify_rows(oracle.interpolation(oracle.biharmonic(g), idx), idx, 12)
    dev = torch.device("cuda:0")
    arrays = dict(rowptr=torch.from_numpy(P.rowptr).to(dev), col=torch.from_numpy(P.col).to(dev),
                  val=torch.from_numpy(P.val).to(dev), W=torch.from_numpy(W).to(dev))
    Zo, tho = oracle.mds_gram(P, W, 3)
    return lib, m.n, idx.size, arrays, (Zo, tho)


def _call(lib, fn, n, l, a, k=3):
    Z = torch.empty((n, k), dtype=torch.float64, device="cuda:0")
    ev = torch.empty((k,), dtype=torch.float64, device="cuda:0")
    o = sb.opts_default()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = getattr(lib, fn)(n, l, _ptr(a["rowptr"]), _ptr(a["col"]), _ptr(a["val"]), _ptr(a["W"]), k, ctypes.byref(o),
                          _ptr(Z), _ptr(ev), stream)
    assert st == 0, lib.sbha_last_error().decode()
    torch.cuda.synchronize()
    return Z.cpu().numpy(), ev.cpu().numpy()


def _gram_err(Z, Zr):
    G1, G2 = Z @ Z.T, Zr @ Zr.T
    return np.abs(G1 - G2).max() / np.abs(G2).max()


def test_static_workspace_matches_sbha_mds_twice(case):
    lib, n, l, a, (Zo, tho) = case
    Zr, evr = _call(lib, "sbha_mds", n, l, a)
    for _ in range(2):  # the fixed workspace keeps the previous call's contents
        Zs, evs = _call(lib, "sbha_mds_static", n, l, a)
        # the same kernels on the same inputs as sbha_mds
        np.testing.assert_allclose(evs, evr, rtol=1e-12)
        assert _gram_err(Zs, Zr) <= 1e-12
        # and the oracle's scaling of the same operator (FP64 bars)
        assert np.max(np.abs(evs - tho) / np.abs(tho)) <= 1e-10
        assert _gram_err(Zs, Zo) <= 1e-10


def test_static_workspace_limits(case):
    lib, n, l, a, _ = case
    Z = torch.empty((n, 3), dtype=torch.float64, device="cuda:0")
    ev = torch.empty((3,), dtype=torch.float64, device="cuda:0")
    # more landmarks than the fixed workspace holds
    st = lib.sbha_mds_static(n, 2000, _ptr(a["rowptr"]), _ptr(a["col"]), _ptr(a["val"]), _ptr(a["W"]), 3, None,
                             _ptr(Z), _ptr(ev), None)
    assert st == 1 and "1024" in lib.sbha_last_error().decode()
    # host arrays are refused
    host_W = a["W"].cpu()
    st = lib.sbha_mds_static(n, l, _ptr(a["rowptr"]), _ptr(a["col"]), _ptr(a["val"]), _ptr(host_W), 3, None,
                             _ptr(Z), _ptr(ev), None)
    assert st == 1 and "device memory" in lib.sbha_last_error().decode()
    # the Lanczos route needs a basis of n-vectors: refused
    o = sb.opts_default(eig_route=sb.EIG_LANCZOS)
    st = lib.sbha_mds_static(n, l, _ptr(a["rowptr"]), _ptr(a["col"]), _ptr(a["val"]), _ptr(a["W"]), 3,
                             ctypes.byref(o), _ptr(Z), _ptr(ev), None)
    assert st == 1 and "Lanczos" in lib.sbha_last_error().decode()
