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
