"""ctypes binding of the arbgpu C ABI (``include/arbgpu.h``): argument marshalling only.

Every computation runs in the CUDA kernels of ``libarbgpu.so``; nothing here computes on the CPU.
If the library has not been built, importing the binding raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libarbgpu.so")

OK = 0
ERR_INVALID = 1
ERR_UNSUPPORTED_VALUE = 2
ERR_WORKSPACE = 3
ERR_CUDA = 4
ERR_TIMEOUT = 5
ERR_LIMIT = 6

ALG_AUTO = 0
ALG_DOT = 1
ALG_BLOCK = 2
MM_COMPLEX_3M = 1

FLAG_SIGN = 1
FLAG_ZERO = 2
FLAG_INF = 4
FLAG_NAN = 8
FLAG_RAD_INF = 16
NSIG_SHIFT = 8


class CBalls(C.Structure):
    _fields_ = [
        ("limbs", C.c_void_p),
        ("limb_stride", C.c_int64),
        ("nlimbs", C.c_int32),
        ("exp", C.c_void_p),
        ("flags", C.c_void_p),
        ("rad_man", C.c_void_p),
        ("rad_exp", C.c_void_p),
        ("count", C.c_int64),
    ]


class CMatmulDesc(C.Structure):
    _fields_ = [("C", CBalls * 2), ("A", CBalls * 2), ("B", CBalls * 2), ("M", C.c_int64),
                ("K", C.c_int64), ("N", C.c_int64), ("lda", C.c_int64), ("ldb", C.c_int64),
                ("ldc", C.c_int64), ("prec", C.c_int32), ("complex_mode", C.c_int32),
                ("alg", C.c_int32), ("flags", C.c_uint32)]


class CTrace(C.Structure):
    _fields_ = [("name", C.c_char_p), ("ms", C.c_float), ("units", C.c_int64),
                ("start_ms", C.c_float)]


class CCalibration(C.Structure):
    _fields_ = [("imad_tops", C.c_double), ("imad_wide_tops", C.c_double),
                ("mma_s8_tops", C.c_double), ("sm_count", C.c_int32),
                ("max_clock_mhz", C.c_double)]


class ArbgpuError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"arbgpu: {what}: status {code} ({status_string(code)})")


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        P = C.POINTER(CBalls)
        L.arbgpu_create.argtypes = [C.POINTER(C.c_void_p), C.c_int]
        L.arbgpu_destroy.argtypes = [vp]
        L.arbgpu_get_status.argtypes = [vp, vp]
        L.arbgpu_status_string.argtypes = [C.c_int]
        L.arbgpu_status_string.restype = C.c_char_p
        L.arbgpu_version.restype = C.c_int
        L.arbgpu_dot.argtypes = [vp, P, P, vp, P, vp, vp, P, vp, vp, vp, vp, i64, i32, i64, C.c_int,
                                 vp, sz, vp]
        L.arbgpu_approx_dot.argtypes = L.arbgpu_dot.argtypes
        L.arbgpu_dot_ex.argtypes = [vp, P, P, vp, P, vp, vp, P, vp, vp, vp, vp, i64, i32, i64,
                                    C.c_int, C.c_uint32, vp, sz, vp]
        L.arbgpu_mat_mul.argtypes = [vp, P, P, P, i64, i64, i64, i64, i64, i64, i32, C.c_int,
                                     C.c_int, C.c_uint32, vp, sz, vp]
        L.arbgpu_mat_mul_workspace_size.argtypes = [vp, i64, i64, i64, i32, i32, i32, C.c_int,
                                                    C.c_int, C.c_uint32, C.POINTER(C.c_size_t)]
        L.arbgpu_int_mat_mul.argtypes = [vp, vp, i32, vp, i32, vp, i32, i64, i64, i64, vp, sz, vp]
        L.arbgpu_int_mat_mul_workspace_size.argtypes = [vp, i32, i32, i64, i64, i64,
                                                        C.POINTER(C.c_size_t)]
        L.arbgpu_int_mat_mul_noalloc.argtypes = [vp, i32, vp, i32, vp, i32, i64, i64, i64, vp, vp]
        L.arbgpu_int_mat_mul_noalloc.restype = C.c_int
        L.arbgpu_mat_mul_batched.argtypes = [vp, C.POINTER(CMatmulDesc), i32, vp, sz, vp]
        L.arbgpu_mat_mul_batched.restype = C.c_int
        L.arbgpu_mat_mul_batched_workspace_size.argtypes = [vp, C.POINTER(CMatmulDesc), i32,
                                                            C.POINTER(C.c_size_t)]
        L.arbgpu_mat_mul_batched_workspace_size.restype = C.c_int
        L.arbgpu_last_plans.argtypes = [vp, vp, i64, C.POINTER(C.c_int64)]
        L.arbgpu_reserve.argtypes = [vp, i32, i64]
        L.arbgpu_calibrate.argtypes = [vp, C.POINTER(CCalibration)]
        L.arbgpu_set_autotune.argtypes = [vp, C.c_int]
        L.arbgpu_autotune_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                            C.POINTER(C.c_int64)]
        L.arbgpu_autotune_alg_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                                C.POINTER(C.c_int64)]
        L.arbgpu_series_exp.argtypes = [vp, P, P, i64, i64, i32, vp, sz, vp]
        L.arbgpu_series_exp_workspace_size.argtypes = [vp, i64, i64, i32, C.POINTER(C.c_size_t)]
        L.arbgpu_launch_count.argtypes = [vp, C.POINTER(C.c_int64)]
        L.arbgpu_trace_enable.argtypes = [vp, C.c_int]
        L.arbgpu_trace_read.argtypes = [vp, C.POINTER(CTrace), i32, C.POINTER(C.c_int32)]
        for name in ("arbgpu_launch_count", "arbgpu_trace_enable", "arbgpu_trace_read",
                     "arbgpu_last_plans", "arbgpu_reserve", "arbgpu_calibrate",
                     "arbgpu_set_autotune", "arbgpu_autotune_stats",
                     "arbgpu_autotune_alg_stats", "arbgpu_series_exp",
                     "arbgpu_series_exp_workspace_size",
                     "arbgpu_create", "arbgpu_destroy", "arbgpu_get_status", "arbgpu_dot",
                     "arbgpu_approx_dot", "arbgpu_dot_ex",
                     "arbgpu_mat_mul", "arbgpu_mat_mul_workspace_size", "arbgpu_int_mat_mul",
                     "arbgpu_int_mat_mul_workspace_size"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def status_string(code) -> str:
    try:
        return lib().arbgpu_status_string(int(code)).decode()
    except Exception:
        return "?"


def exported_symbols():
    """Names the shared library must export (every function declared in include/arbgpu.h)."""
    return ["arbgpu_create", "arbgpu_destroy", "arbgpu_get_status", "arbgpu_status_string",
            "arbgpu_version", "arbgpu_launch_count", "arbgpu_trace_enable", "arbgpu_trace_read",
            "arbgpu_dot", "arbgpu_approx_dot", "arbgpu_dot_ex", "arbgpu_mat_mul",
            "arbgpu_mat_mul_workspace_size",
            "arbgpu_int_mat_mul", "arbgpu_int_mat_mul_workspace_size",
            "arbgpu_int_mat_mul_noalloc", "arbgpu_mat_mul_batched",
            "arbgpu_mat_mul_batched_workspace_size", "arbgpu_last_plans", "arbgpu_reserve",
            "arbgpu_series_exp", "arbgpu_series_exp_workspace_size", "arbgpu_calibrate",
            "arbgpu_set_autotune", "arbgpu_autotune_stats", "arbgpu_autotune_alg_stats"]
