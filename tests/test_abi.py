"""The C-ABI library builds for sm_103a, loads, and exports what the header declares.

No compute call is made here (these tests run without a GPU)."""
import ctypes as C

import pytest

from paper_1704_05528_gb300 import _lib as L
from paper_1704_05528_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def test_header_declares_the_boundary():
    names = L.header_functions()
    for required in ("svt_complete", "svt_r4svd", "svt_pattern_create", "svt_pattern_destroy",
                     "svt_spmm", "svt_sampled_update", "svt_sampled_update_recycle",
                     "svt_complete_eval",
                     "svt_gaussian_block"):
        assert required in names


def test_every_header_symbol_is_exported(lib):
    names = L.header_functions()
    assert names, "no functions parsed from the header"
    missing = [nm for nm in names if not hasattr(lib, nm)]
    assert not missing, f"symbols declared but not exported: {missing}"
    assert set(names) <= set(L.SIGNATURES), "binding lacks a signature for a header function"


def test_struct_layouts():
    # int32 fields first, then 8-byte fields, as declared in the header
    assert C.sizeof(L.Options) == 10 * 4 + 3 * 8 + 8
    assert C.sizeof(L.IterLog) == 6 * 4 + 7 * 8
    assert C.sizeof(L.Result) == 6 * 4 + 6 * 8


def test_defaults_and_strings(lib):
    o = L.Options()
    lib.svt_default_options(C.byref(o))
    assert (o.t, o.dt, o.n_power, o.r_max) == (-1, 10, 0, 0)
    assert abs(o.beta - 0.95) < 1e-15 and o.precision == L.SVT_FP64
    assert (o.recycle, o.stop, o.core_rows, o.reserved) == (0, 0, -1, 0)
    assert lib.svt_abi_version() == 3
    assert lib.svt_status_string(L.SVT_ERR_DUPLICATE) == b"duplicate observed entry"
    assert lib.svt_status_string(12345) == b"unknown status"


def test_argument_validation_without_gpu(lib):
    o = L.Options()
    lib.svt_default_options(C.byref(o))
    res = L.Result()
    st = lib.svt_complete(0, 5, 0, None, None, None, 1.0, 1.0, 1e-3, 10, C.byref(o), None, None,
                          None, 5, C.byref(res), None, 0, None, 0)
    assert st == L.SVT_ERR_ARG and res.status == L.SVT_ERR_ARG
    st = lib.svt_complete(4, 5, 0, None, None, None, -1.0, 1.0, 1e-3, 10, C.byref(o), None, None,
                          None, 5, C.byref(res), None, 0, None, 0)
    assert st == L.SVT_ERR_ARG
    assert b"tau" in lib.svt_last_error()
    h = C.c_void_p()
    assert lib.svt_pattern_create(-1, 3, 0, None, None, None, C.byref(h)) == L.SVT_ERR_ARG
    for field, value, word in (("recycle", 3, b"recycle"), ("stop", 2, b"stop")):
        bad = L.Options()
        lib.svt_default_options(C.byref(bad))
        setattr(bad, field, value)
        st = lib.svt_complete(4, 5, 0, None, None, None, 1.0, 1.0, 1e-3, 10, C.byref(bad), None,
                              None, None, 5, C.byref(res), None, 0, None, 0)
        assert st == L.SVT_ERR_ARG and word in lib.svt_last_error()
    st = lib.svt_complete_eval(4, 5, 0, None, None, None, 3, None, None, None, 1.0, 1.0, 1e-3, 10,
                               C.byref(o), None, None, None, 5, C.byref(res), None, 0, None, 0)
    assert st == L.SVT_ERR_ARG and b"evaluation" in lib.svt_last_error()
    sums = (C.c_double * 3)()
    assert lib.svt_sampled_update_recycle(None, L.SVT_FP64, None, 4, 4, None, 4, 2, None, None, 1.0,
                                          None, 4, sums, None) == L.SVT_ERR_ARG


def test_unrolled_params_defaults_and_validation(lib):
    assert C.sizeof(L.UnrolledParams) == 4 * 4 + 2 * 8
    assert C.sizeof(L.UnrolledInfo) == 8 * 4 + 3 * 8
    up = L.UnrolledParams()
    lib.svt_unrolled_default_params(C.byref(up), L.SVT_FP64)
    assert (up.steps, up.checkpoint_every, up.cg_maxit, up.ritz_maxit) == (20, 5, 1000, 100)
    assert up.cg_tol == 1e-10 and up.ritz_tol == 1e-11
    lib.svt_unrolled_default_params(C.byref(up), L.SVT_MIXED_FP32)
    assert up.cg_tol == 1e-6 and up.ritz_tol == 2e-6
    o = L.Options()
    lib.svt_default_options(C.byref(o))
    info = L.UnrolledInfo()
    # rejected before any device work: no held-out set, then a bad checkpoint interval
    idx = (C.c_int32 * 1)(0)
    val = (C.c_double * 1)(1.0)
    st = lib.svt_unrolled_grad(2, 2, 1, idx, idx, val, 0, idx, idx, val, 1.0, 1.0, None, C.byref(o),
                               None, None, None, C.byref(info))
    assert st == L.SVT_ERR_ARG
    lib.svt_unrolled_default_params(C.byref(up), L.SVT_FP64)
    up.checkpoint_every = 0
    st = lib.svt_unrolled_grad(2, 2, 1, idx, idx, val, 1, idx, idx, val, 1.0, 1.0, C.byref(up),
                               C.byref(o), None, None, None, C.byref(info))
    assert st == L.SVT_ERR_ARG and b"checkpoint_every" in lib.svt_last_error()


def test_workspace_sizes_and_a_short_workspace_is_refused_before_any_work(lib):
    """svt_workspace_size grows with the problem and the evaluation set, includes the dense
    core's panel for binary32 solves with a core, and a workspace below it is refused with
    SVT_ERR_ARG before anything is queued (the pointer is never touched)."""
    o = L.Options()
    lib.svt_default_options(C.byref(o))
    o.r_max = 100
    small = lib.svt_workspace_size(1000, 800, 50_000, 0, 100, C.byref(o))
    big = lib.svt_workspace_size(1000, 800, 200_000, 0, 100, C.byref(o))
    ev = lib.svt_workspace_size(1000, 800, 50_000, 5_000, 100, C.byref(o))
    assert 0 < small < big and small < ev
    o.precision = L.SVT_MIXED_FP32
    o.core_rows = 0
    plain = lib.svt_workspace_size(1000, 800, 200_000, 0, 100, C.byref(o))
    o.core_rows = 256
    cored = lib.svt_workspace_size(1000, 800, 200_000, 0, 100, C.byref(o))
    assert cored >= plain + 2 * 800 * 256 * 4  # the core's A and Y panels
    assert lib.svt_r4svd_workspace_size(1000, 800, 50_000, C.byref(o)) > 0
    bad = L.Options()
    lib.svt_default_options(C.byref(bad))
    bad.dt = 0
    assert lib.svt_workspace_size(1000, 800, 50_000, 0, 100, C.byref(bad)) == 0
    res = L.Result()
    rows = (C.c_int32 * 4)(0, 1, 2, 3)
    vals = (C.c_double * 4)(1.0, 2.0, 3.0, 4.0)
    fake = C.c_void_p(0x1000)  # never dereferenced: the size check comes first
    st = lib.svt_complete(4, 4, 4, rows, rows, vals, 1.0, 1.0, 1e-3, 10, C.byref(o), None, None,
                          None, 4, C.byref(res), None, 0, fake, 1024)
    assert st == L.SVT_ERR_ARG and b"workspace" in lib.svt_last_error()
