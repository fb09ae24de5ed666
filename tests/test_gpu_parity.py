"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars:
  * edge graph, lengths, cotangent weights A, lumped mass D, weight sums V and the
    biharmonic operator M: bit-exact (both sides form every term in the same order with
    correctly rounded operations);
  * landmark ids, min-distance fields, geodesic distances and W: bit-exact (both sides
    add the same edge lengths left to right along shortest paths);
  * operator pattern: bit-exact, except in rows where the oracle's p-th and (p+1)-th
    magnitudes are closer than twice the solve's error bound (counted and reported);
  * operator values, FP64: max_i |P_gpu - P_oracle| <= 1e-10 max_i |P_oracle| in every
    column j (the oracle's columns are the exactly rounded solutions of Eq. 3), with the solve
    run to cg_rtol = 1e-12 (factored) or 1e-13 (direct CG on M_uu, whose error stays in the
    smooth modes and is larger for the same residual); at these tolerances the refinement
    residuals are formed in double-double.  Mixed precision (FP32 inner solves refined on the FP64
    residual to the same cg_rtol): 1e-8 of the column maximum.  Both also stay within the
    rigorous bound rtol ||b_j|| / lambda_min(M_uu) + 1e-12;
  * eigenvalues 1e-10 relative and embeddings through Z Z^T (unique when the top-k
    eigenvalues are separated from the rest) 1e-10 of max |Z Z^T| in FP64; 1e-8 and 1e-6
    with mixed-precision operators.
Every test prints the largest error it measured (tests/_report.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import meshgen  # noqa: E402
import oracle  # noqa: E402
import paper_1705_10887_gb300 as sb  # noqa: E402
from tests._report import col_rel_err, gram_rel_err, report  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

# several tiles and ragged edges: l not a multiple of 32, l > 512 (two chunks), open and closed meshes
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
        idx, mind = oracle.fps(g, l, 0)
        W = oracle.landmark_block(g, idx)
        M = oracle.biharmonic(g)
        Pd = oracle.interpolation(M, idx)
        _cache[name] = dict(mesh=m, l=l, p=p, g=g, idx=idx, mind=mind, W=W, M=M, Pd=Pd)
    return _cache[name]


def error_bounds(r, rtol):
    """Per-column bound rtol ||b_j|| / lambda_min(M_uu) on the FP64 solve error."""
    M = r["M"].todense()
    unk = np.setdiff1d(np.arange(M.shape[0]), r["idx"])
    Muu, Mub = M[np.ix_(unk, unk)], M[np.ix_(unk, r["idx"])]
    lam = np.linalg.eigvalsh(Muu)[0]
    return rtol * np.linalg.norm(Mub, axis=0) / lam + 1e-12


# FP64 runs tighten cg_rtol so that the solve error is well inside the 1e-10 bar.  Residuals of an
# exactly rounded P are about 5e-14 of ||b|| on these meshes (the biharmonic rows cancel), so 1e-12
# leaves room; the direct solver needs the tighter 1e-13 for its forward error.
RTOL_FP64 = 1e-12
RTOL_FP64_DIRECT = 1e-13
FP64_BAR, MIXED_BAR = 1e-10, 1e-8


@pytest.mark.parametrize("name", list(CASES))
def test_mesh_quantities_bit_exact(name):
    r = ref(name)
    m, g = r["mesh"], r["g"]
    rowptr, col, ln, A, D, V = (t.cpu().numpy() for t in sb.mesh_graph(cuda(m.xyz), cuda(m.faces)))
    assert np.array_equal(rowptr, g.rowptr) and np.array_equal(col, g.col)
    assert np.array_equal(ln, g.length)
    assert np.array_equal(A, g.A)
    assert np.array_equal(D, g.D)
    assert np.array_equal(V, oracle.weight_sums(g))
    mr, mc, mv = (t.cpu().numpy() for t in sb.biharmonic(cuda(m.xyz), cuda(m.faces)))
    M = r["M"]
    assert np.array_equal(mr, M.rowptr) and np.array_equal(mc, M.col)
    assert np.array_equal(mv, M.val)
    report("mesh_quantities", case=name, edges=int(col.size), nnz_M=int(mc.size), bit_exact=True)


@pytest.mark.parametrize("name", list(CASES))
def test_landmarks_bit_exact(name):
    r = ref(name)
    m = r["mesh"]
    idx, mind = sb.landmarks(cuda(m.xyz), cuda(m.faces), r["l"], 0, return_mind=True)
    assert np.array_equal(idx.cpu().numpy(), r["idx"])
    assert np.array_equal(mind.cpu().numpy(), r["mind"])


@pytest.mark.parametrize("name", list(CASES))
def test_geodesics_bit_exact(name):
    r = ref(name)
    m = r["mesh"]
    src = np.array([0, m.n // 2, m.n - 1, 7], np.int32)
    D = sb.geodesics(cuda(m.xyz), cuda(m.faces), cuda(src))
    assert np.array_equal(D.cpu().numpy(), oracle.geodesics(r["g"], src))
    tgt = np.array([3, 1, m.n - 2], np.int32)
    D = sb.geodesics(cuda(m.xyz), cuda(m.faces), cuda(src), cuda(tgt))
    assert np.array_equal(D.cpu().numpy(), oracle.geodesics(r["g"], src, tgt))
    W = sb.landmark_distances(cuda(m.xyz), cuda(m.faces), cuda(r["idx"]))
    assert np.array_equal(W.cpu().numpy(), r["W"])


def _csr_dense(rowptr, col, val, n, l):
    rp, c, v = (t.cpu().numpy() if hasattr(t, "cpu") else t for t in (rowptr, col, val))
    out = np.zeros((n, l))
    mask = np.zeros((n, l), bool)
    for i in range(n):
        s, e = rp[i], rp[i + 1]
        assert np.all(np.diff(c[s:e]) > 0)
        out[i, c[s:e]] = v[s:e]
        mask[i, c[s:e]] = True
    return out, mask


def check_operator(r, P, mask, S, Smask, bound, bar):
    n, l = r["Pd"].shape
    # landmark rows exactly e_j
    assert np.array_equal(P[r["idx"]], np.eye(l))
    # values: every kept GPU entry within the bar of its column's largest entry, and within the
    # rigorous bound of the dense oracle value
    err = col_rel_err(P, r["Pd"], mask)
    assert err <= bar, f"largest error {err:.3e} of a column's maximum (bar {bar:.0e})"
    diff = np.abs(P - r["Pd"]) * mask
    viol = diff > bound[None, :]
    assert not viol.any(), f"max excess {np.max(diff - bound[None, :])}"
    # pattern: equal except at certified near-ties
    bad_rows = np.nonzero(np.any(mask != Smask, axis=1))[0]
    unk = np.setdiff1d(np.arange(n), r["idx"])
    for i in bad_rows:
        a = np.sort(np.abs(r["Pd"][i]))[::-1]
        keep = mask[i].sum()
        margin = a[keep - 1] - a[keep] if keep < l else np.inf
        assert margin <= 2 * bound.max(), f"row {i}: pattern differs with margin {margin}"
    return len(bad_rows), unk.size, err


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [sb.PREC_FP64, sb.PREC_FP32_REFINE])
@pytest.mark.parametrize("solver", [sb.SOLVER_FACTORED, sb.SOLVER_DIRECT])
def test_operator_rows(name, prec, solver):
    r = ref(name)
    m, l, p = r["mesh"], r["l"], r["p"]
    rtol = (RTOL_FP64_DIRECT if solver == sb.SOLVER_DIRECT else RTOL_FP64) if prec == sb.PREC_FP64 else 1e-11
    o = sb.opts_default(precision=prec, cg_rtol=rtol, solver=solver)
    rowptr, col, val = sb.operator(cuda(m.xyz), cuda(m.faces), cuda(r["idx"]), p, o)
    st = sb.last_stats()
    assert st["cg_max_rel_residual"] <= rtol * 1.0001
    P, mask = _csr_dense(rowptr, col, val, m.n, l)
    S = oracle.sparsify_rows(r["Pd"], r["idx"], p)
    Sd = S.todense()
    Smask = np.zeros_like(mask)
    for i in range(m.n):
        Smask[i, S.col[S.rowptr[i] : S.rowptr[i + 1]]] = True
    assert int(rowptr[-1]) == l + (m.n - l) * min(p, l)
    bar = FP64_BAR if prec == sb.PREC_FP64 else MIXED_BAR
    bad, total, err = check_operator(r, P, mask, Sd, Smask, error_bounds(r, rtol), bar)
    report("operator_rows", case=name, precision=int(prec), solver=int(solver), cg_rtol=rtol, max_rel=err,
           bar=bar, near_tie_rows=bad, residual=st["cg_max_rel_residual"])
    assert bad <= max(1, total // 1000)


@pytest.mark.parametrize("name", ["icosphere3", "torus60x40"])
def test_operator_columns(name):
    r = ref(name)
    m, l, p = r["mesh"], r["l"], r["p"]
    rtol = RTOL_FP64
    o = sb.opts_default(sparsify_mode=sb.SPARSIFY_COLS, cg_rtol=rtol)
    rowptr, col, val = sb.operator(cuda(m.xyz), cuda(m.faces), cuda(r["idx"]), p, o)
    P, mask = _csr_dense(rowptr, col, val, m.n, l)
    S = oracle.sparsify_cols(r["Pd"], r["idx"], p)
    Smask = np.zeros_like(mask)
    for i in range(m.n):
        Smask[i, S.col[S.rowptr[i] : S.rowptr[i + 1]]] = True
    pc = oracle.column_mode_p(m.n, l, p)
    assert int(rowptr[-1]) == l + l * pc
    bound = error_bounds(r, rtol)
    assert np.array_equal(P[r["idx"]], np.eye(l))
    assert not (np.abs(P - r["Pd"]) * mask > bound[None, :]).any()
    err = col_rel_err(P, r["Pd"], mask)
    report("operator_columns", case=name, max_rel=err, bar=FP64_BAR)
    assert err <= FP64_BAR
    # pattern by columns, near-ties excepted
    for j in range(l):
        if np.array_equal(mask[:, j], Smask[:, j]):
            continue
        unk = np.setdiff1d(np.arange(m.n), r["idx"])
        a = np.sort(np.abs(r["Pd"][unk, j]))[::-1]
        assert a[pc - 1] - a[pc] <= 2 * bound[j]


@pytest.mark.parametrize("name", list(CASES))
def test_mds_on_oracle_operator(name):
    r = ref(name)
    S = oracle.sparsify_rows(r["Pd"], r["idx"], r["p"])
    Zo, tho = oracle.mds_gram(S, r["W"], 3)
    Z, ev = sb.mds(r["mesh"].n, cuda(S.rowptr), cuda(S.col), cuda(S.val), cuda(r["W"]), 3)
    st = sb.last_stats()
    ev = ev.cpu().numpy()
    Z = Z.cpu().numpy()
    ev_err = float(np.max(np.abs(ev - tho) / np.abs(tho)))
    z_err = gram_rel_err(Z, Zo)
    report("mds_on_oracle_operator", case=name, eval_rel=ev_err, zzt_rel=z_err, ritz_residual=st["eig_residual"],
           iterations=st["eig_iterations"])
    assert ev_err <= 1e-10 and z_err <= 1e-10
    # the sign rule: largest-magnitude entry of each column positive
    for q in range(3):
        i = int(np.argmax(np.abs(Z[:, q])))
        assert Z[i, q] > 0
    assert st["eig_residual"] <= sb.opts_default().eig_tol


@pytest.mark.parametrize("name", ["icosphere3", "torus60x40", "patch40"])
@pytest.mark.parametrize("prec", [sb.PREC_FP64, sb.PREC_FP32_REFINE])
def test_embed_end_to_end(name, prec):
    r = ref(name)
    m, l, p = r["mesh"], r["l"], r["p"]
    ro = oracle.sbmds(m.xyz, m.faces, l, p, 3, 0)
    fp64 = prec == sb.PREC_FP64
    o = sb.opts_default(precision=prec, cg_rtol=RTOL_FP64 if fp64 else 1e-11)
    Z, ev, idx = sb.embed(cuda(m.xyz), cuda(m.faces), l, p, 3, 0, o)
    assert np.array_equal(idx.cpu().numpy(), ro.idx)
    ev = ev.cpu().numpy()
    ev_err = float(np.max(np.abs(ev - ro.theta) / np.abs(ro.theta)))
    z_err = gram_rel_err(Z.cpu().numpy(), ro.Z)
    report("embed_end_to_end", case=name, precision=int(prec), eval_rel=ev_err, zzt_rel=z_err)
    assert ev_err <= (1e-10 if fp64 else 1e-8)
    assert z_err <= (1e-10 if fp64 else 1e-6)


def test_host_buffers_match_device_buffers():
    r = ref("torus60x40")
    m = r["mesh"]
    Zh, evh, idxh = sb.embed(m.xyz, m.faces, r["l"], r["p"], 3)
    Zd, evd, idxd = sb.embed(cuda(m.xyz), cuda(m.faces), r["l"], r["p"], 3)
    assert isinstance(Zh, np.ndarray)
    assert np.array_equal(idxh, idxd.cpu().numpy())
    np.testing.assert_allclose(evh, evd.cpu().numpy(), rtol=1e-12)


def test_degenerate_sizes():
    m = meshgen.icosphere(1, noise=0.01, seed=2)  # n = 42
    g = oracle.mesh_operators(m.xyz, m.faces)
    # l = n: every vertex a landmark, P = I
    idx, _ = oracle.fps(g, m.n, 0)
    rowptr, col, val = sb.operator(m.xyz, m.faces, idx, 4)
    assert np.array_equal(rowptr, np.arange(m.n + 1))
    assert np.array_equal(col, np.argsort(idx))  # row idx[j] holds column j
    assert np.all(val == 1.0)
    P = np.zeros((m.n, m.n))
    P[np.arange(m.n), col] = val
    assert np.array_equal(P[idx], np.eye(m.n))
    # l = 1: every row of P is 1 (constants are biharmonic), kept once per row
    rowptr, col, val = sb.operator(m.xyz, m.faces, np.array([5], np.int32), 3)
    assert np.array_equal(rowptr, np.arange(m.n + 1))
    np.testing.assert_allclose(val, 1.0, atol=1e-9)
    # p_row > l: rows keep all l entries
    idx, _ = oracle.fps(g, 6, 0)
    rowptr, col, val = sb.operator(m.xyz, m.faces, idx, 20)
    assert rowptr[-1] == 6 + (m.n - 6) * 6


def test_errors():
    m = meshgen.icosphere(1)
    with pytest.raises(sb.SbhaError) as e:
        sb.operator(m.xyz, m.faces, np.array([1, 1, 2], np.int32), 2)
    assert e.value.status == 1
    bad = m.faces.copy()
    bad[3, 2] = m.n + 4
    with pytest.raises(sb.SbhaError) as e:
        sb.landmarks(m.xyz, bad, 3)
    assert e.value.status == 1
    a, b = meshgen.icosphere(1, seed=1), meshgen.icosphere(1, seed=2)
    xyz = np.concatenate([a.xyz, b.xyz + 4.0])
    faces = np.concatenate([a.faces, b.faces + a.n])
    with pytest.raises(sb.SbhaError) as e:
        sb.landmarks(xyz, faces, 3)
    assert e.value.status == 2
    with pytest.raises(sb.SbhaError) as e:
        sb.geodesics(m.xyz, m.faces, np.array([0, m.n], np.int32))
    assert e.value.status == 1
