"""ctypes loader of ``libkifmm_m2l.so`` (the C ABI of include/kifmm_m2l.h).

Argument marshalling only.  The library is loaded from this package's
directory; when it is missing the import fails loudly (there is no CPU or
Python fallback for the translation).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkifmm_m2l.so")

KIFMM_OK = 0
KIFMM_ERR_TIMEOUT = -5
ERR_NAMES = {
    -1: "KIFMM_ERR_INVALID_ARG",
    -2: "KIFMM_ERR_UNSUPPORTED",
    -3: "KIFMM_ERR_CUDA",
    -4: "KIFMM_ERR_OOM",
    -5: "KIFMM_ERR_TIMEOUT",
    -6: "KIFMM_ERR_STATE",
}

PREC = {"fp32": 0, "bf16": 1, "split3": 2, "split6": 3, "f16x3": 4}
N_OFFSETS = 316

# every symbol include/kifmm_m2l.h declares
EXPORTED = (
    "kifmm_m2l_precompute", "kifmm_m2l_destroy", "kifmm_m2l_plan_rank", "kifmm_m2l_set_level",
    "kifmm_m2l_level_pairs", "kifmm_m2l_apply", "kifmm_m2l_apply_adjoint", "kifmm_m2l_apply_dense", "kifmm_m2l_apply_dense_tc",
    "kifmm_m2l_apply_noalloc", "kifmm_m2l_apply_levels", "kifmm_m2l_apply_levels_adjoint",
    "kifmm_m2l_apply_levels_host",
    "kifmm_m2l_apply_batch",
    "kifmm_m2l_set_stage2", "kifmm_m2l_stage2_ranks", "kifmm_m2l_stage2_host",
    "kifmm_m2l_sync", "kifmm_m2l_set_wait_limit", "kifmm_m2l_profile_enable", "kifmm_m2l_profile_read", "kifmm_m2l_autotune",
    "kifmm_m2l_factors_host", "kifmm_m2l_pairs_host", "kifmm_m2l_last_error", "kifmm_m2l_version",
    "kifmm_fmm_create", "kifmm_fmm_evaluate", "kifmm_fmm_set_normals", "kifmm_fmm_info", "kifmm_fmm_destroy", "kifmm_m2l_pass_ops_host",
)


class Params(ctypes.Structure):
    _fields_ = [("kernel_id", ctypes.c_int), ("p", ctypes.c_int), ("eps", ctypes.c_double),
                ("d", ctypes.c_double), ("precision", ctypes.c_int), ("kappa", ctypes.c_double),
                ("box_halfwidth", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("n_chunk", ctypes.c_int), ("contiguous", ctypes.c_int), ("variant", ctypes.c_int),
                ("core_ms", ctypes.c_double), ("from_cache", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("instance", ctypes.c_int), ("level_lo", ctypes.c_int),
                ("level_hi", ctypes.c_int), ("nrhs", ctypes.c_int), ("q_up", ctypes.c_void_p),
                ("p_down", ctypes.c_void_p), ("beta", ctypes.c_float)]


class KifmmError(RuntimeError):
    def __init__(self, func: str, status: int, message: str):
        super().__init__(f"{func} failed: {ERR_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load (once) and return the library; raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_1211_2517_gb300.build` "
            "(the M2L has no fallback implementation)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_double
    pint, pi64 = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)
    sig = {
        "kifmm_m2l_precompute": [ctypes.POINTER(Params), ctypes.POINTER(vp)],
        "kifmm_m2l_destroy": [vp],
        "kifmm_m2l_plan_rank": [vp, pint, pint, pint],
        "kifmm_m2l_set_level": [vp, i32, i32, f64, i32, vp],
        "kifmm_m2l_level_pairs": [vp, i32, i32, pi64],
        "kifmm_m2l_apply": [vp, i32, i32, i32, vp, vp, f32, vp],
        "kifmm_m2l_apply_adjoint": [vp, i32, i32, i32, vp, vp, f32, vp],
        "kifmm_m2l_apply_dense": [vp, i32, i32, i32, vp, vp, f32, vp],
        "kifmm_m2l_apply_dense_tc": [vp, i32, i32, i32, vp, vp, f32, vp],
        "kifmm_m2l_apply_noalloc": [vp, i32, i32, i32, vp, vp, f32, vp],
        "kifmm_m2l_apply_levels": [vp, i32, i32, i32, i32, vp, vp, f32, vp],
        "kifmm_m2l_apply_levels_adjoint": [vp, i32, i32, i32, i32, vp, vp, f32, vp],
        "kifmm_m2l_apply_levels_host": [vp, i32, i32, i32, i32, vp, vp, f32, vp],
        "kifmm_m2l_apply_batch": [i32, ctypes.POINTER(BatchItem), i32, vp],
        "kifmm_m2l_sync": [vp, vp],
        "kifmm_m2l_set_wait_limit": [vp, ctypes.c_ulonglong],
        "kifmm_m2l_profile_enable": [vp, i32],
        "kifmm_m2l_profile_read": [vp, ctypes.POINTER(ctypes.c_double), pi64],
        "kifmm_m2l_autotune": [vp, i32, i32, i32, i32, vp, vp, i32, ctypes.POINTER(TuneResult), vp],
        "kifmm_m2l_set_stage2": [vp, ctypes.c_double],
        "kifmm_m2l_stage2_ranks": [vp, pint],
        "kifmm_m2l_stage2_host": [ctypes.POINTER(Params), ctypes.c_double, pint, vp],
        "kifmm_m2l_factors_host": [ctypes.POINTER(Params), pint, pint, vp, vp, vp],
        "kifmm_m2l_pairs_host": [i32, i32, vp, pi64, vp, vp, vp],
        "kifmm_fmm_create": [vp, i64, vp, i32, vp, f64, ctypes.POINTER(vp)],
        "kifmm_fmm_evaluate": [vp, vp, vp, i32, vp],
        "kifmm_fmm_set_normals": [vp, vp],
        "kifmm_fmm_info": [vp, pint, pi64, pi64, pi64, pi64],
        "kifmm_fmm_destroy": [vp],
        "kifmm_m2l_pass_ops_host": [ctypes.POINTER(Params), f64, pint, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = i32
    L.kifmm_m2l_last_error.argtypes = []
    L.kifmm_m2l_last_error.restype = ctypes.c_char_p
    L.kifmm_m2l_version.argtypes = []
    L.kifmm_m2l_version.restype = ctypes.c_char_p
    _lib = L
    return L


def check(func: str, status: int) -> None:
    if status != KIFMM_OK:
        msg = lib().kifmm_m2l_last_error().decode(errors="replace")
        raise KifmmError(func, status, msg)


def call(name: str, *args) -> None:
    check(name, getattr(lib(), name)(*args))
