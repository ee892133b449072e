"""ctypes declarations of the C-ABI in include/qg.h (argument marshalling only).

The shared library is the in-tree build ``_build/libqg.so``; importing the
binding without it raises immediately.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqg.so")

QG_OK = 0
QG_ERR_ARG = -1
QG_ERR_CUDA = -2
QG_ERR_NONFINITE = -3
QG_ERR_OOM = -4
QG_ERR_TIMEOUT = -5
QG_ERR_UNSUPPORTED = -6
QG_ERR_BOUNDS = -7
QG_FP64 = 0
QG_FP32 = 1
QG_SCHEME_RK3_EXACT = 0
QG_SCHEME_AB2CN = 1
QG_NONE, QG_SMAG, QG_LEITH, QG_DSMAG, QG_DLEITH = 0, 1, 2, 3, 4
KERNEL_CLASSES = ("row_stage", "col_reduce", "col_stage", "row_brinkman", "col_curl", "row_sponge", "col_final",
                  "other", "adj_row", "adj_col", "adj_pointwise")

ERROR_NAMES = {
    QG_ERR_ARG: "QG_ERR_ARG", QG_ERR_CUDA: "QG_ERR_CUDA", QG_ERR_NONFINITE: "QG_ERR_NONFINITE",
    QG_ERR_OOM: "QG_ERR_OOM", QG_ERR_TIMEOUT: "QG_ERR_TIMEOUT", QG_ERR_UNSUPPORTED: "QG_ERR_UNSUPPORTED",
    QG_ERR_BOUNDS: "QG_ERR_BOUNDS",
}


class qg_grid(C.Structure):
    _fields_ = [("n", C.c_int32), ("precision", C.c_int32), ("L", C.c_double)]


class qg_closure(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("c", C.c_double), ("test_ratio", C.c_double)]


class qg_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("nu", C.c_double), ("mu", C.c_double), ("eta", C.c_double),
                ("sponge_rate", C.c_double), ("scheme", C.c_int32), ("reserved", C.c_int32)]


class qg_diag(C.Structure):
    _fields_ = [("t", C.c_double), ("energy", C.c_double), ("enstrophy", C.c_double), ("coeff", C.c_double),
                ("max_abs_omega", C.c_double), ("step", C.c_int64), ("finite", C.c_int32), ("reserved", C.c_int32)]


class qg_member(C.Structure):
    _fields_ = [("grid", qg_grid), ("closure", qg_closure), ("params", qg_params), ("beta", C.c_double),
                ("U", C.c_double), ("mask", C.POINTER(C.c_double)), ("sponge", C.POINTER(C.c_double))]


DP = C.POINTER(C.c_double)

# name -> (restype, argtypes): every symbol include/qg.h declares
SIGNATURES = {
    "qg_create": (C.c_int, [C.POINTER(qg_grid), C.c_double, C.c_double, DP, DP, C.POINTER(qg_closure),
                            C.POINTER(qg_params), C.c_void_p, C.POINTER(C.c_void_p)]),
    "qg_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "qg_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "qg_step": (C.c_int, [C.c_void_p, C.c_int32]),
    "qg_sync": (C.c_int, [C.c_void_p]),
    "qg_stream": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "qg_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(qg_diag)]),
    "qg_destroy": (None, [C.c_void_p]),
    "qg_sgs_apriori": (C.c_int, [DP, C.c_int32, C.c_int32, C.c_double, DP, DP, C.POINTER(qg_closure),
                                 C.POINTER(qg_params), C.c_double, C.c_double, C.c_int32, DP, DP, DP, DP]),
    "qg_grid_filter": (C.c_int, [DP, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int32, DP]),
    "qg_series_compare": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.c_int32,
                                    C.c_int32, C.c_int32, C.c_void_p, DP, DP, DP, C.POINTER(C.c_int32), DP]),
    "qg_ensemble_create": (C.c_int, [C.POINTER(qg_member), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "qg_ensemble_handle": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "qg_ensemble_step": (C.c_int, [C.c_void_p, C.c_int32]),
    "qg_ensemble_sync": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "qg_ensemble_config": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), DP]),
    "qg_ensemble_destroy": (None, [C.c_void_p]),
    "qg_step_vjp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, DP]),
    "qg_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "qg_kernel_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double), C.c_int32]),
    "qg_field_stats_static": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_void_p, C.c_void_p]),
    "qg_probe_fma_rate": (C.c_int, [C.c_int32, DP, DP]),
    "qg_last_error": (C.c_char_p, []),
    "qg_version": (C.c_char_p, []),
}

_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Load libqg and declare every entry point; raises if the build is missing.

    The environment variable QG_LIB selects another build of the library.
    """
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("QG_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libqg is not built ({path} missing): run __graft_entry__.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class QGError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str) -> int:
    if code != QG_OK:
        raise QGError(code, where, load().qg_last_error().decode())
    return code
