"""Host-side tests of the C ABI (no GPU needed).

The library must load and export every entry point include/spkadd.h declares,
and the argument checks of spkadd_plan must reject bad calls before touching
CUDA (so they run on a machine without a GPU).
"""
import ctypes
import os
import re

import pytest

import paper_2112_10223_gb300 as spk
from paper_2112_10223_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return spk.library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "spkadd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spkadd_[a-z_]+)\s*\(", text)))


def test_header_declares_the_four_phases():
    names = declared_functions()
    for f in ("spkadd_plan", "spkadd_symbolic", "spkadd_numeric", "spkadd_destroy"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"


def test_only_the_c_abi_is_exported(lib):
    out = os.popen(f"nm -D --defined-only {_build.LIB_PATH}").read()
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert exported == set(declared_functions())


def test_status_strings_and_version(lib):
    for code, name in spk.STATUS.items():
        assert spk.spkadd_status_string(code).startswith(name)
    assert lib.spkadd_version() >= 100


def test_default_options(lib):
    o = spk.default_options()
    assert (o.validate, o.warp_max, o.cta_max, o.window_max, o.sort_mode, o.input_order, o.block_accumulator) == \
        (0, 512, 4096, 4096, 0, 0, 0)


def _csc(m=4, n=3, nnz=0, cp=1, ri=0, va=0):
    c = spk.CSC()
    c.m, c.n, c.nnz = m, n, nnz
    c.col_ptr, c.row_idx, c.val = cp or None, ri or None, va or None
    return c


def _plan(lib, arr, k=None, dtype=1, opt=None):
    h = ctypes.c_void_p(123)
    st = lib.spkadd_plan(ctypes.byref(h), len(arr) if k is None else k, arr if arr else None, dtype, None,
                         ctypes.byref(opt) if opt is not None else None)
    return st, h


@pytest.mark.parametrize("case,expect", [
    ("k0", 1), ("null_A", 1), ("bad_dtype", 1), ("negative_m", 1), ("shape_m", 2), ("shape_n", 2),
    ("m_overflow", 5), ("nnz_overflow", 5), ("null_colptr", 1), ("null_rows", 1), ("null_vals", 1),
    ("k_too_large", 10),
])
def test_plan_rejects_bad_arguments_without_cuda(lib, case, expect):
    arr = (spk.CSC * 2)(_csc(), _csc())
    k, dtype = None, 1
    if case == "k0":
        k = 0
    elif case == "null_A":
        arr = None
        k = 2
    elif case == "bad_dtype":
        dtype = 7
    elif case == "negative_m":
        arr[1].m = -1
    elif case == "shape_m":
        arr[1].m = 5
    elif case == "shape_n":
        arr[1].n = 4
    elif case == "m_overflow":
        arr[0].m = arr[1].m = 2 ** 31
    elif case == "nnz_overflow":
        arr[1].nnz = 2 ** 31
    elif case == "null_colptr":
        arr[1].col_ptr = None
    elif case == "null_rows":
        arr[1].nnz, arr[1].val = 5, 8
    elif case == "null_vals":
        arr[1].nnz, arr[1].row_idx = 5, 8
    elif case == "k_too_large":
        k = 65537
    st, h = _plan(lib, arr, k=k, dtype=dtype)
    assert st == expect, spk.spkadd_status_string(st)
    assert not h.value  # handle set to NULL on failure


def test_plan_null_handle_pointer(lib):
    arr = (spk.CSC * 1)(_csc())
    assert lib.spkadd_plan(None, 1, arr, 1, None, None) == 1


@pytest.mark.parametrize("field,value", [
    ("warp_max", 0), ("warp_max", 513), ("cta_max", 4097), ("window_max", 1000), ("window_max", 5000),
    ("sort_mode", 3), ("sort_mode", -1), ("input_order", 2), ("input_order", -1),
    ("block_accumulator", 3), ("block_accumulator", -1),
])
def test_plan_rejects_bad_options(lib, field, value):
    o = spk.default_options(**{field: value})
    arr = (spk.CSC * 1)(_csc())
    st, _ = _plan(lib, arr, opt=o)
    assert st == 1


def test_cta_max_below_warp_max_rejected(lib):
    o = spk.default_options(warp_max=256, cta_max=100)
    st, _ = _plan(lib, (spk.CSC * 1)(_csc()), opt=o)
    assert st == 1


def test_calls_on_null_handle(lib):
    n = ctypes.c_int64()
    assert lib.spkadd_symbolic(None, ctypes.byref(n)) == 1
    assert lib.spkadd_numeric(None, None, None, None) == 1
    assert lib.spkadd_get_info(None, None) == 1
    assert lib.spkadd_destroy(None) == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(spk, "_lib", None)
    monkeypatch.setattr(spk, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(spk.SpkaddError):
        spk.library()


def _batch_plan(lib, problems, dtypes=None, count=None):
    """problems: list of lists of CSC; returns (status, handle)."""
    arrs = [(spk.CSC * len(p))(*p) for p in problems]
    ks = (ctypes.c_int * max(1, len(problems)))(*[len(p) for p in problems])
    ptrs = (ctypes.c_void_p * max(1, len(problems)))(*[ctypes.cast(a, ctypes.c_void_p) for a in arrs])
    dts = (ctypes.c_int * max(1, len(problems)))(*(dtypes or [1] * len(problems)))
    h = ctypes.c_void_p(123)
    st = lib.spkadd_batch_plan(ctypes.byref(h), len(problems) if count is None else count,
                               ctypes.cast(ks, ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p),
                               ctypes.cast(dts, ctypes.c_void_p), None, None)
    return st, h


@pytest.mark.parametrize("case,expect", [
    ("count0", 1), ("k0", 1), ("shape_inside_problem", 2), ("bad_dtype", 1), ("second_problem_overflow", 5),
    ("total_columns_overflow", 5),
])
def test_batch_plan_rejects_bad_arguments_without_cuda(lib, case, expect):
    # Problems may differ in shape from each other; inside one they may not.
    problems = [[_csc(m=4, n=3), _csc(m=4, n=3)], [_csc(m=9, n=5)]]
    dtypes, count = [1, 0], None
    if case == "count0":
        count = 0
    elif case == "k0":
        problems[1] = []
    elif case == "shape_inside_problem":
        problems[0][1].n = 4
    elif case == "bad_dtype":
        dtypes = [1, 3]
    elif case == "second_problem_overflow":
        problems[1][0].nnz = 2 ** 31
    elif case == "total_columns_overflow":
        problems[0][0].n = problems[0][1].n = 2 ** 30
        problems[1][0].n = 2 ** 30
    st, h = _batch_plan(lib, problems, dtypes=dtypes, count=count)
    assert st == expect, spk.spkadd_status_string(st)
    assert not h.value


def test_batch_calls_on_null_handle(lib):
    n = (ctypes.c_int64 * 1)()
    assert lib.spkadd_batch_symbolic(None, ctypes.cast(n, ctypes.c_void_p)) == 1
    assert lib.spkadd_batch_numeric(None, None, None, None) == 1


def test_batch_descriptor_layout_matches_the_header():
    # The binding packs descriptors with numpy; the record must be spkadd_csc.
    assert spk._CSC_NP.itemsize == ctypes.sizeof(spk.CSC) == 48
    assert [spk._CSC_NP.fields[f][1] for f in ("m", "n", "nnz", "col_ptr", "row_idx", "val")] == \
        [getattr(spk.CSC, f).offset for f in ("m", "n", "nnz", "col_ptr", "row_idx", "val")]


@pytest.mark.parametrize("m,n,dtype,expect", [
    (-1, 4, 1, "SPKADD_ERR_INVALID_ARG"), (4, -1, 1, "SPKADD_ERR_INVALID_ARG"), (4, 4, 2, "SPKADD_ERR_INVALID_ARG"),
    (2**31, 4, 1, "SPKADD_ERR_OVERFLOW"), (4, 2**31 - 1, 0, "SPKADD_ERR_OVERFLOW"),
])
def test_stream_create_rejects_bad_arguments_without_cuda(lib, m, n, dtype, expect):
    s = ctypes.c_void_p(1)
    st = lib.spkadd_stream_create(ctypes.byref(s), m, n, dtype, None, None)
    assert spk.STATUS[st] == expect
    assert not s.value  # *s cleared on failure


def test_stream_create_rejects_bad_options_and_null_out(lib):
    o = spk.default_options(window_max=5000)
    s = ctypes.c_void_p()
    assert spk.STATUS[lib.spkadd_stream_create(ctypes.byref(s), 4, 4, 1, None, ctypes.byref(o))] == \
        "SPKADD_ERR_INVALID_ARG"
    assert spk.STATUS[lib.spkadd_stream_create(None, 4, 4, 1, None, None)] == "SPKADD_ERR_INVALID_ARG"


def test_stream_calls_on_null_stream_handle(lib):
    n = ctypes.c_int64()
    assert spk.STATUS[lib.spkadd_stream_add(None, 1, (spk.CSC * 1)())] == "SPKADD_ERR_INVALID_ARG"
    assert spk.STATUS[lib.spkadd_stream_query(None, ctypes.byref(n), None, None)] == "SPKADD_ERR_INVALID_ARG"
    assert spk.STATUS[lib.spkadd_stream_view(None, None)] == "SPKADD_ERR_INVALID_ARG"
    assert spk.STATUS[lib.spkadd_stream_result(None, None, None, None)] == "SPKADD_ERR_INVALID_ARG"
    assert lib.spkadd_stream_destroy(None) == 0


def test_stream_class_rejects_bad_dtype_before_cuda(lib):
    import torch

    with pytest.raises(TypeError):
        spk.SpkaddStream(4, 4, dtype=torch.int32)
