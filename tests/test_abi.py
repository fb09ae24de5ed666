"""The C ABI library loads and exports every entry point declared in include/sbha.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1705_10887_gb300 as sb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sb.build()
    return sb.library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sbha.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sbha_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = declared_functions()
    assert len(names) >= 10
    bound = {n for n, _, _ in sb.SIGNATURES}
    for name in names:
        assert hasattr(lib, name), f"{name} missing from libsbha.so"
        assert name in bound, f"{name} has no Python binding"


def test_defaults_and_version(lib):
    o = sb.opts_default()
    assert o.precision == sb.PREC_FP64 and o.sparsify_mode == sb.SPARSIFY_ROWS
    assert 0 < o.cg_rtol < 1e-6 and o.cg_max_iter > 0 and o.oversample >= 0
    assert "sm_103a" in sb.version()


def test_size_query_without_gpu(lib):
    # nnz = l + (n - l) * min(p_row, l) in row mode; l + l * round((n-l) p_row / l) in column mode
    assert sb.operator_nnz(642, 32, 8) == 32 + 610 * 8
    assert sb.operator_nnz(50000, 500, 16) == 500 + 49500 * 16
    assert sb.operator_nnz(100, 10, 20) == 10 + 90 * 10
    o = sb.opts_default(sparsify_mode=sb.SPARSIFY_COLS)
    assert sb.operator_nnz(642, 32, 8, o) == 32 + 32 * 153


def test_argument_errors_are_reported_without_gpu(lib):
    m = sb.Mesh(10, 5, None, None)
    idx = (ctypes.c_int32 * 1)()
    st = lib.sbha_landmarks(ctypes.byref(m), 0, 0, ctypes.cast(idx, ctypes.c_void_p), None, None)
    assert st == 1
    assert "l must be" in lib.sbha_last_error().decode()
    st = lib.sbha_operator(ctypes.byref(m), ctypes.cast(idx, ctypes.c_void_p), 1, 0, None, None, None, None, 0, None,
                           None)
    assert st == 1 and "p_row" in lib.sbha_last_error().decode()
    o = sb.opts_default(precision=7)
    with pytest.raises(sb.SbhaError):
        sb.operator_nnz(100, 10, 4, o)


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of include/sbha.h, from a small C program built with gcc."""
    import shutil
    import subprocess
    import tempfile

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = [f'printf("%zu\\n", sizeof({struct}));']
    lines += [f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    src = "#include <stddef.h>\n#include <stdio.h>\n#include \"sbha.h\"\nint main(void) {\n" + "\n".join(lines) + \
        "\nreturn 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c_file, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(c_file, "w") as f:
            f.write(src)
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), c_file, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("struct, cls", [("sbha_mesh", sb.Mesh), ("sbha_graph", sb.Graph), ("sbha_opts", sb.Opts),
                                         ("sbha_stats", sb.Stats)])
def test_struct_layouts_match_the_header(struct, cls):
    names = [f for f, _ in cls._fields_]
    size, offsets = _c_layout(struct, names)
    assert ctypes.sizeof(cls) == size, f"{struct}: ctypes size {ctypes.sizeof(cls)} vs C {size}"
    for name, off in zip(names, offsets):
        assert getattr(cls, name).offset == off, f"{struct}.{name}: ctypes offset {getattr(cls, name).offset} vs C {off}"


def test_prototype_arity_matches_the_bindings():
    src = open(os.path.join(ROOT, "include", "sbha.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = dict(re.findall(r"\b(sbha_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", src))
    for name, _, argtypes in sb.SIGNATURES:
        params = protos[name].strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert n == len(argtypes), f"{name}: header has {n} parameters, binding {len(argtypes)}"


def test_next_row_entry_points_reject_bad_arguments_without_gpu(lib):
    m = sb.Mesh(10, 5, None, None)
    idx = (ctypes.c_int32 * 2)(0, 1)
    pidx = ctypes.cast(idx, ctypes.c_void_p)
    out = (ctypes.c_double * 4)()
    pout = ctypes.cast(out, ctypes.c_void_p)
    assert lib.sbha_heat_geodesics(ctypes.byref(m), pidx, 0, 1.0, None, pout, None) == 1
    assert lib.sbha_fmds_operator(ctypes.byref(m), pidx, 0, 50.0, None, pout, None) == 1
    assert "l must be" in lib.sbha_last_error().decode()
    g = sb.Graph(10, None, None, None)
    assert lib.sbha_graph_operator(ctypes.byref(g), pidx, 2, 0, None, None, None, None, 0, None, None) == 1
    assert "p_row" in lib.sbha_last_error().decode()
    assert lib.sbha_bha_error(0, 2, None, None, None, None, 0, None, None, 0, pout, pout, None) == 1
    bad = sb.opts_default()
    bad.spmm_chunk_rows = 48
    with pytest.raises(sb.SbhaError):
        sb.operator_nnz(100, 10, 4, bad)


@pytest.mark.parametrize("field, bad", [("spmm_variant", 5), ("spmm_variant", -1), ("spmm_pipeline_depth", 3),
                                        ("spmm_chunk_rows", 48), ("cg_graph", 2), ("mlp_pilot_cols", 513),
                                        ("mlp_pilot_cols", -1), ("fault_inject", 9), ("dense_mode", 3),
                                        ("eig_route", 2), ("cg_rtol", 0.0), ("eig_tol", -1.0)])
def test_option_values_are_checked_without_gpu(lib, field, bad):
    """Every option is validated before any device work: an out-of-range value is SBHA_EINVAL with a message."""
    with pytest.raises(sb.SbhaError) as e:
        sb.operator_nnz(100, 10, 4, sb.opts_default(**{field: bad}))
    assert e.value.status == 1 and lib.sbha_last_error().decode()


@pytest.mark.parametrize("field, good", [("spmm_variant", sb.SPMM_TMA), ("spmm_variant", sb.SPMM_PIPELINED),
                                         ("spmm_pipeline_depth", 4), ("spmm_chunk_rows", -1), ("cg_graph", 0),
                                         ("mlp_pilot_cols", 256), ("fault_inject", sb.FAULT_MLP_NAN)])
def test_accepted_option_values_without_gpu(field, good):
    """The documented values of the options pass validation (the size query touches no device)."""
    assert sb.operator_nnz(100, 10, 4, sb.opts_default(**{field: good})) > 0
