"""ctypes declarations of the C ABI in include/svt_gb300.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "svt_gb300.h")
LIB_PATH = os.path.join(HERE, "libsvt_gb300.so")

SVT_OK, SVT_NOT_CONVERGED = 0, 1
SVT_ERR_ARG, SVT_ERR_INDEX, SVT_ERR_DUPLICATE, SVT_ERR_CUDA = -1, -2, -3, -4
SVT_ERR_NUMERIC, SVT_ERR_UNSUPPORTED = -6, -8
SVT_FP64, SVT_MIXED_FP32 = 0, 1


class Options(C.Structure):
    _fields_ = [("t", C.c_int32), ("dt", C.c_int32), ("n_power", C.c_int32),
                ("r_max", C.c_int32), ("power_steps", C.c_int32), ("precision", C.c_int32),
                ("recycle", C.c_int32), ("stop", C.c_int32), ("core_rows", C.c_int32),
                ("reserved", C.c_int32), ("beta", C.c_double), ("eps_thr0", C.c_double), ("seed", C.c_uint64),
                ("stream", C.c_void_p)]


class IterLog(C.Structure):
    _fields_ = [("iter", C.c_int32), ("r", C.c_int32), ("k", C.c_int32), ("blocks", C.c_int32),
                ("cooled", C.c_int32), ("exhausted", C.c_int32), ("eps", C.c_double),
                ("eps_thr", C.c_double), ("rel_residual", C.c_double), ("mae", C.c_double),
                ("sigma_max", C.c_double), ("seconds", C.c_double), ("mae_eval", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("k", C.c_int32), ("r", C.c_int32),
                ("k0", C.c_int32), ("log_len", C.c_int32), ("rel_residual", C.c_double),
                ("mae", C.c_double), ("spec_norm", C.c_double), ("eps_thr", C.c_double),
                ("seconds_pattern", C.c_double), ("seconds_total", C.c_double)]


class UnrolledParams(C.Structure):
    _fields_ = [("steps", C.c_int32), ("checkpoint_every", C.c_int32), ("cg_maxit", C.c_int32),
                ("ritz_maxit", C.c_int32), ("cg_tol", C.c_double), ("ritz_tol", C.c_double)]


class UnrolledInfo(C.Structure):
    _fields_ = [("k0", C.c_int32), ("k_final", C.c_int32), ("r_final", C.c_int32),
                ("cg_iters", C.c_int32), ("cg_capped", C.c_int32), ("ritz_steps", C.c_int32),
                ("ritz_capped", C.c_int32), ("ritz_grown", C.c_int32),
                ("loss", C.c_double), ("seconds_forward", C.c_double), ("seconds_total", C.c_double)]


_P = C.c_void_p
_I32, _I64, _U32, _U64, _D = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
_PI32 = C.POINTER(C.c_int32)
_PD = C.POINTER(C.c_double)

SIGNATURES = {
    "svt_abi_version": (C.c_int, []),
    "svt_default_options": (None, [C.POINTER(Options)]),
    "svt_status_string": (C.c_char_p, [C.c_int]),
    "svt_last_error": (C.c_char_p, []),
    "svt_pattern_create": (C.c_int, [_I64, _I64, _I64, _P, _P, _P, C.POINTER(_P)]),
    "svt_pattern_destroy": (None, [_P]),
    "svt_pattern_nnz": (_I64, [_P]),
    "svt_pattern_export": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "svt_gaussian_block": (C.c_int, [_U64, _U32, _U32, _I64, _I32, _P, _I64, _P]),
    "svt_spmm": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _I64, _I32, _P, _I64, _P]),
    "svt_spmm_noalloc": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _I64, _I32, _P, _I64, _P]),
    "svt_sampled_update": (C.c_int, [_P, C.c_int, _P, _I64, _P, _I64, _I32, _P, _P, _D, _PD, _P]),
    "svt_sampled_update_recycle": (C.c_int, [_P, C.c_int, _P, _I64, _I32, _P, _I64, _I32, _P, _P,
                                             _D, _P, _I64, _PD, _P]),
    "svt_r4svd": (C.c_int, [_P, _P, _P, _I64, _I32, _D, _U32, C.POINTER(Options), _P, _I64, _P,
                            _P, _I64, _PI32, _PD, _PI32, _P, C.c_size_t]),
    "svt_workspace_size": (C.c_size_t, [_I64, _I64, _I64, _I64, _I32, C.POINTER(Options)]),
    "svt_r4svd_workspace_size": (C.c_size_t, [_I64, _I64, _I64, C.POINTER(Options)]),
    "svt_profile_enable": (None, [C.c_int]),
    "svt_profile_reset": (None, []),
    "svt_launch_count": (C.c_int64, []),
    "svt_profile_read": (C.c_int, [C.c_int, _P, C.POINTER(C.c_int64), _PD, _PD]),
    "svt_unrolled_default_params": (None, [C.POINTER(UnrolledParams), C.c_int]),
    "svt_unrolled_grad": (C.c_int, [_I64, _I64, _I64, _P, _P, _P, _I64, _P, _P, _P, _D, _D,
                                     C.POINTER(UnrolledParams), C.POINTER(Options), _P, _P, _P,
                                     C.POINTER(UnrolledInfo)]),
    "svt_complete": (C.c_int, [_I64, _I64, _I64, _P, _P, _P, _D, _D, _D, _I32,
                               C.POINTER(Options), _P, _P, _P, _I32, C.POINTER(Result),
                               C.POINTER(IterLog), _I32, _P, C.c_size_t]),
    "svt_complete_eval": (C.c_int, [_I64, _I64, _I64, _P, _P, _P, _I64, _P, _P, _P, _D, _D, _D, _I32,
                                    C.POINTER(Options), _P, _P, _P, _I32, C.POINTER(Result),
                                    C.POINTER(IterLog), _I32, _P, C.c_size_t]),
    "svt_test_set_grid_wait_limit": (C.c_uint, [C.c_uint]),
    "svt_unrolled_forward": (C.c_int, [_I64, _I64, _I64, _P, _P, _P, _I64, _P, _P, _D, _D,
                                        C.POINTER(UnrolledParams), C.POINTER(Options), _P,
                                        C.POINTER(UnrolledInfo), C.POINTER(_P)]),
    "svt_unrolled_backward": (C.c_int, [_P, _P, _P, _P, C.POINTER(UnrolledInfo)]),
    "svt_unrolled_tape_destroy": (None, [_P]),
}


def header_functions(path: str = HEADER):
    """Names of the functions declared in the public header."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(svt_[a-z0-9_]+)\s*\(", text)) - {"svt_status"})


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (building it first if it is missing) and declare signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing and could not be built")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
