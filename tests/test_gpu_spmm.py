"""The block-CG product kernels (register gather, pipelined gather, staged tiles, TMA gather) give the
operator of the oracle, with unknowns in locality order."""
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


@pytest.mark.parametrize("variant", [sb.SPMM_GATHER, sb.SPMM_STAGED, sb.SPMM_PIPELINED, sb.SPMM_TMA])
@pytest.mark.parametrize("solver, precision", [(sb.SOLVER_FACTORED, sb.PREC_FP64), (sb.SOLVER_FACTORED, sb.PREC_FP32_REFINE),
                                               (sb.SOLVER_DIRECT, sb.PREC_FP64), (sb.SOLVER_DIRECT, sb.PREC_FP32_REFINE)])
def test_variants_match_oracle(variant, solver, precision):
    # 3000 unknowns: 24 row tiles of 128 (47 of 64), a ragged last tile; two-ring pattern for the
    # direct solver, whose 64-row tiles partly exceed the TMA stage and take its global-memory path
    m = meshgen.torus(60, 51, 1.0, 0.3, 0.2, seed=11)
    g = oracle.mesh_operators(m.xyz, m.faces)
    l = 40
    idx, _ = oracle.fps(g, l, 0)
    Pd = oracle.interpolation(oracle.biharmonic(g), idx)
    xyz, faces, didx = (torch.from_numpy(a).cuda() for a in (m.xyz, m.faces, idx))
    rtol = 1e-10
    o = sb.opts_default(spmm_variant=variant, solver=solver, precision=precision, cg_rtol=rtol, chunk_cols=32)
    rowptr, col, val = sb.operator(xyz, faces, didx, 8, o)
    st = sb.last_stats()
    assert st["cg_max_rel_residual"] <= rtol
    if variant == sb.SPMM_STAGED:
        assert st["spmm_tiles"] == (m.n - l + 127) // 128
        if solver == sb.SOLVER_FACTORED:  # one-ring halos fit the stage; two-ring ones (M_uu) partly fall back
            assert st["spmm_tiles_staged"] == st["spmm_tiles"]
    else:
        assert st["spmm_tiles"] == 0
    if variant == sb.SPMM_TMA and precision == sb.PREC_FP32_REFINE:
        assert st["spmm_tma"] == 1
        ntiles = (m.n - l + 63) // 64
        if solver == sb.SOLVER_FACTORED:
            assert st["spmm_gather_tiles_staged"] == ntiles
        else:
            assert st["spmm_gather_tiles_staged"] < ntiles
    else:
        assert st["spmm_tma"] == 0
    rp, cc, vv = rowptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    rows = np.repeat(np.arange(m.n), np.diff(rp))
    assert np.abs(vv - Pd[rows, cc]).max() < 1e-7
    # the kept entries are the largest of each row (up to near-ties at the solver tolerance)
    for v in range(0, m.n, 97):
        if v in set(idx.tolist()):
            continue
        kept = np.sort(np.abs(vv[rp[v]:rp[v + 1]]))
        full = np.sort(np.abs(Pd[v]))[::-1][:8]
        assert np.abs(np.sort(full) - kept).max() < 1e-7


def test_variant_rejected():
    m = meshgen.icosphere(2, 0.01, 0)
    with pytest.raises(sb.SbhaError):
        sb.operator(m.xyz, m.faces, np.arange(8, dtype=np.int32), 4, sb.opts_default(spmm_variant=7))


def test_launch_shape_autotuned_once_per_shape():
    """The gather kernels time their candidate launch shapes on a matrix shape's first product and keep
    the fastest; a second call with the same shape reuses it, and the operator is the oracle's."""
    m = meshgen.torus(64, 50, 1.0, 0.3, 0.2, seed=21)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 33, 0)
    xyz, faces, didx = (torch.from_numpy(a).cuda() for a in (m.xyz, m.faces, idx))
    o = sb.opts_default(precision=sb.PREC_FP32_REFINE, cg_rtol=1e-10)
    sb.operator(xyz, faces, didx, 8, o)
    st = sb.last_stats()
    assert st["spmm_chunk_rows"] in (16, 32, 64) and st["spmm_tuned_us"] > 0.0  # contiguous only when asked for
    shapes = st["spmm_tuned_shapes"]
    assert shapes >= 1
    rowptr, col, val = sb.operator(xyz, faces, didx, 8, o)
    st2 = sb.last_stats()
    assert st2["spmm_tuned_shapes"] == shapes and st2["spmm_chunk_rows"] == st["spmm_chunk_rows"]
    Pd = oracle.interpolation(oracle.biharmonic(g), idx)
    rp, c, v = (t.cpu().numpy() for t in (rowptr, col, val))
    rows = np.repeat(np.arange(m.n), np.diff(rp))
    assert np.abs(v - Pd[rows, c]).max() < 1e-7


def test_fixed_launch_shapes_give_the_same_operator():
    m = meshgen.torus(40, 30, 1.0, 0.3, 0.2, seed=22)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 24, 0)
    xyz, faces, didx = (torch.from_numpy(a).cuda() for a in (m.xyz, m.faces, idx))
    ref = sb.operator(xyz, faces, didx, 8, sb.opts_default(cg_rtol=1e-11))[2].cpu().numpy()
    for chunk in (-1, 16, 32, 64):
        v = sb.operator(xyz, faces, didx, 8, sb.opts_default(cg_rtol=1e-11, spmm_chunk_rows=chunk))[2].cpu().numpy()
        assert sb.last_stats()["spmm_chunk_rows"] == max(chunk, 0)
        assert np.abs(v - ref).max() <= 1e-9 * np.abs(ref).max()
    with pytest.raises(sb.SbhaError) as e:
        sb.operator(xyz, faces, didx, 8, sb.opts_default(spmm_chunk_rows=48))
    assert e.value.status == 1


@pytest.mark.parametrize("depth", [2, 4])
def test_pipelined_gather_depths(depth):
    """The pipelined gather (cp.async ring of 2 or 4 rows per warp) in the learned + mixed configuration,
    which also runs the fused direction update through it: the operator equals the register gather's
    to the solver tolerance and the oracle's, and the stats report the depth that ran."""
    m = meshgen.torus(70, 48, 1.0, 0.3, 0.2, seed=23)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 70, 0)
    xyz, faces, didx = (torch.from_numpy(a).cuda() for a in (m.xyz, m.faces, idx))
    base = dict(precision=sb.PREC_FP32_REFINE, precond=sb.PRECOND_MLP, cg_rtol=1e-11, spmm_chunk_rows=32)
    ref = sb.operator(xyz, faces, didx, 8, sb.opts_default(spmm_variant=sb.SPMM_GATHER, **base))
    assert sb.last_stats()["spmm_pipeline_depth"] == 0
    got = sb.operator(xyz, faces, didx, 8, sb.opts_default(spmm_variant=sb.SPMM_PIPELINED,
                                                          spmm_pipeline_depth=depth, **base))
    st = sb.last_stats()
    assert st["spmm_pipeline_depth"] == depth and st["mlp_trained"] == 1
    assert st["cg_max_rel_residual"] <= 1e-11 * 1.0001
    assert np.array_equal(ref[0].cpu().numpy(), got[0].cpu().numpy())
    v0, v1 = ref[2].cpu().numpy(), got[2].cpu().numpy()
    assert np.abs(v1 - v0).max() <= 1e-9 * np.abs(v0).max()
    Pd = oracle.interpolation(oracle.biharmonic(g), idx)
    rp, c = got[0].cpu().numpy(), got[1].cpu().numpy()
    rows = np.repeat(np.arange(m.n), np.diff(rp))
    assert np.abs(v1 - Pd[rows, c]).max() <= 1e-8 * np.abs(Pd).max()


@pytest.mark.parametrize("precision, precond", [(sb.PREC_FP64, sb.PRECOND_JACOBI),
                                                (sb.PREC_FP32_REFINE, sb.PRECOND_MLP)])
def test_device_decided_cg_loop(precision, precond):
    """Block-CG solves finished as one CUDA graph whose WHILE node the device decides (cg_graph = 1, the
    default) give the operator of the host-checked batches (cg_graph = 0), and both the oracle's; a stream is
    needed for the graph (the legacy default stream keeps the host loop)."""
    m = meshgen.torus(60, 44, 1.0, 0.3, 0.2, seed=31)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 48, 0)
    Pd = oracle.interpolation(oracle.biharmonic(g), idx)
    xyz, faces, didx = (torch.from_numpy(a).cuda() for a in (m.xyz, m.faces, idx))
    out = {}
    with torch.cuda.stream(torch.cuda.Stream()):
        for gflag in (0, 1):
            o = sb.opts_default(precision=precision, precond=precond, cg_rtol=1e-11, cg_graph=gflag)
            rp, c, v = sb.operator(xyz, faces, didx, 10, o)
            st = sb.last_stats()
            assert st["cg_max_rel_residual"] <= 1e-11 * 1.0001
            out[gflag] = (rp.cpu().numpy(), c.cpu().numpy(), v.cpu().numpy(), st["cg_iterations"])
    assert np.array_equal(out[0][0], out[1][0])
    for gflag in (0, 1):
        rp, c, v, _ = out[gflag]
        rows = np.repeat(np.arange(m.n), np.diff(rp))
        assert np.abs(v - Pd[rows, c]).max() <= 1e-9 * np.abs(Pd).max()
    # the graph runs two iterations per pass: at most one more per solve than the host loop stops at
    assert abs(out[1][3] - out[0][3]) <= max(8, out[0][3] // 20)


def test_tma_gather_product_full_width():
    """The TMA gather product over 16 column blocks (four groups per tile) with the learned preconditioner,
    whose products all go through it, and a second chunk whose padding columns leave blocks inactive
    from the start: the operator equals the register gather's (the products sum every row in the same
    order) to the solver tolerance, and sampled columns equal the oracle's exactly rounded ones."""
    m = meshgen.torus(80, 61, 1.0, 0.3, 0.2, seed=24)
    g = oracle.mesh_operators(m.xyz, m.faces)
    l = 520
    idx, _ = oracle.fps(g, l, 0)
    xyz, faces, didx = (torch.from_numpy(a).cuda() for a in (m.xyz, m.faces, idx))
    base = dict(precision=sb.PREC_FP32_REFINE, precond=sb.PRECOND_MLP, cg_rtol=1e-11)
    ref = sb.operator(xyz, faces, didx, 16, sb.opts_default(spmm_variant=sb.SPMM_GATHER, **base))
    assert sb.last_stats()["spmm_tma"] == 0
    got = sb.operator(xyz, faces, didx, 16, sb.opts_default(spmm_variant=sb.SPMM_TMA, **base))
    st = sb.last_stats()
    assert st["spmm_tma"] == 1 and st["mlp_trained"] == 1 and st["chunk_cols"] == 512
    assert st["spmm_gather_tiles_staged"] == (m.n - l + 63) // 64
    assert st["cg_max_rel_residual"] <= 1e-11 * 1.0001
    assert np.array_equal(ref[0].cpu().numpy(), got[0].cpu().numpy())
    v0, v1 = ref[2].cpu().numpy(), got[2].cpu().numpy()
    assert np.abs(v1 - v0).max() <= 1e-9 * np.abs(v0).max()
    cols = np.arange(3, l, 37)
    Ps = oracle.interpolation(oracle.biharmonic(g), idx, cols=cols)
    rp, c = got[0].cpu().numpy(), got[1].cpu().numpy()
    rows = np.repeat(np.arange(m.n), np.diff(rp))
    pos = {int(j): q for q, j in enumerate(cols)}
    sel = np.array([int(cc) in pos for cc in c])
    want = Ps[rows[sel], [pos[int(cc)] for cc in c[sel]]]
    assert sel.sum() > 0 and np.abs(v1[sel] - want).max() <= 1e-9 * np.abs(Ps).max()


def test_tma_wait_timeout_is_an_error():
    """A bounded wait of the TMA gather product that runs out (the wait limit set to zero) makes the
    solve return SBHA_ETIMEOUT after the kernel has waited for its own gathers; the next call with
    the default limit is correct."""
    m = meshgen.torus(40, 30, 1.0, 0.3, 0.2, seed=25)
    g = oracle.mesh_operators(m.xyz, m.faces)
    idx, _ = oracle.fps(g, 24, 0)
    xyz, faces, didx = (torch.from_numpy(a).cuda() for a in (m.xyz, m.faces, idx))
    o = sb.opts_default(spmm_variant=sb.SPMM_TMA, precision=sb.PREC_FP32_REFINE, cg_rtol=1e-10)
    prev = sb.set_wait_limit(0)
    try:
        with pytest.raises(sb.SbhaError) as e:
            sb.operator(xyz, faces, didx, 8, o)
        assert e.value.status == 6
    finally:
        sb.set_wait_limit(-1)
    assert prev > 0
    rowptr, col, val = sb.operator(xyz, faces, didx, 8, o)
    assert sb.last_stats()["spmm_tma"] == 1
    Pd = oracle.interpolation(oracle.biharmonic(g), idx)
    rp, c, v = (t.cpu().numpy() for t in (rowptr, col, val))
    rows = np.repeat(np.arange(m.n), np.diff(rp))
    assert np.abs(v - Pd[rows, c]).max() < 1e-7
