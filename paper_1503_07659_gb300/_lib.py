"""ctypes binding of libsemax (include/semax.h).

Argument marshalling only: every step of the operator runs in the library's
CUDA kernels.  There is no CPU or PyTorch fallback: if the shared library is
missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsemax.so")

SEMAX_OK = 0
SEMAX_ETIMEOUT = -6
SEMAX_F64, SEMAX_F32 = 0, 1
SEMAX_PLAN_F64X, SEMAX_PLAN_F64TC, SEMAX_PLAN_F64TC_PREPARED = 1, 2, 4
SEMAX_PCG_F64X, SEMAX_PCG_F64TC, SEMAX_PCG_MIXED = 1, 2, 4

STATUS_NAMES = {
    0: "SEMAX_OK", -1: "SEMAX_EINVAL", -2: "SEMAX_EUNSUPPORTED_N", -3: "SEMAX_EALIGN",
    -4: "SEMAX_EALIAS", -5: "SEMAX_ECUDA", -6: "SEMAX_ETIMEOUT", -7: "SEMAX_ENOPLAN",
    -8: "SEMAX_EWORKSPACE", -9: "SEMAX_EIO",
}

# every symbol include/semax.h declares
EXPORTS = (
    "sem_ax", "sem_ax_helmholtz", "sem_ax_helmholtz_f64tc", "sem_ax_f64x", "sem_ax_f64tc", "sem_ax_f64tc_status", "sem_ax_f64tc_prepare_size",
    "sem_ax_f64tc_prepare", "sem_ax_f64tc_prepared", "sem_ax_f64tc_prepared_status", "sem_ax_f32", "sem_ax_bf16x3", "sem_ax_f16x3", "sem_ax_bf16x3_geo",
    "sem_ax_batched_workspace_size", "sem_ax_batched",
    "sem_ax_plan_create", "sem_ax_plan_exec", "sem_ax_plan_destroy", "sem_ax_plan_status", "sem_ax_plan_config",
    "semax_gs_create", "semax_gs_apply", "semax_gs_destroy", "sem_ax_diag",
    "sem_pcg_create", "sem_pcg_solve", "sem_pcg_destroy",
    "semax_reduce_workspace_size", "semax_reduce", "semax_reduce_noalloc",
    "semax_strerror", "semax_last_cuda_error", "semax_set_wait_polls", "semax_fma_probe",
)


class SemaxError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.semax_strerror(status).decode() if _lib is not None else ""
        cuda = f" (cudaError {_lib.semax_last_cuda_error()})" if status == -5 and _lib is not None else ""
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}{cuda}")


class semax_group(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("E", ctypes.c_int64), ("u", ctypes.c_void_p),
                ("G", ctypes.c_void_p), ("D", ctypes.c_void_p), ("w", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsemax is not built ({LIB_PATH} missing); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    i64, i32, vp, sz = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
    sig = {
        "sem_ax": [i64, i32, vp, vp, vp, vp, vp],
        "sem_ax_f64x": [i64, i32, vp, vp, vp, vp, vp],
        "sem_ax_f64tc": [i64, i32, vp, vp, vp, vp, vp],
        "sem_ax_f64tc_status": [i64, i32, vp, vp, vp, vp, vp, vp],
        "sem_ax_f64tc_prepared_status": [i64, i32, vp, vp, vp, vp, vp, vp],
        "sem_ax_f64tc_prepare_size": [i64, i32, ctypes.POINTER(sz)],
        "sem_ax_f64tc_prepare": [i64, i32, vp, vp, vp],
        "sem_ax_f64tc_prepared": [i64, i32, vp, vp, vp, vp, vp],
        "sem_ax_helmholtz": [i64, i32, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp],
        "sem_ax_helmholtz_f64tc": [i64, i32, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp],
        "sem_ax_f32": [i64, i32, vp, vp, vp, vp, vp, vp],
        "sem_ax_bf16x3": [i64, i32, vp, vp, vp, vp, vp, i32, vp],
        "sem_ax_f16x3": [i64, i32, vp, vp, vp, vp, vp, vp],
        "sem_ax_bf16x3_geo": [i64, i32, vp, vp, vp, vp, vp, i32, vp],
        "sem_ax_batched_workspace_size": [vp, i32, ctypes.POINTER(sz)],
        "sem_ax_batched": [vp, i32, vp, sz, vp],
        "sem_ax_plan_create": [ctypes.POINTER(vp), vp, i32, i32, ctypes.c_char_p, i32],
        "sem_ax_plan_exec": [vp, vp],
        "sem_ax_plan_destroy": [vp],
        "sem_ax_plan_status": [vp, vp],
        "sem_ax_plan_config": [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "semax_gs_create": [ctypes.POINTER(vp), i64, vp, i64, vp],
        "semax_gs_apply": [vp, vp, i32, vp],
        "semax_gs_destroy": [vp],
        "sem_ax_diag": [i64, i32, vp, vp, vp, vp],
        "sem_pcg_create": [ctypes.POINTER(vp), i64, i32, vp, vp, vp, i32],
        "sem_pcg_solve": [vp, vp, vp, i32, ctypes.c_double, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double), vp],
        "sem_pcg_destroy": [vp],
        "semax_reduce_workspace_size": [i64, ctypes.POINTER(sz)],
        "semax_reduce": [i64, vp, i32, vp, i32, vp, vp, sz, vp],
        "semax_reduce_noalloc": [i64, vp, i32, vp, i32, vp, vp],
        "semax_strerror": [i32],
        "semax_last_cuda_error": [],
        "semax_set_wait_polls": [i32],
        "semax_fma_probe": [i32, i32, i32, vp, ctypes.POINTER(ctypes.c_double), vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)  # raises AttributeError if the library lacks a declared symbol
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "semax_strerror" else ctypes.c_int
    return lib


_lib = None
_lib = _load()


def lib():
    return _lib


def check(status: int, where: str) -> None:
    if status != SEMAX_OK:
        raise SemaxError(status, where)
