"""ctypes declarations of the C ABI in include/mm.h.

This module only loads the in-tree ``lib/libmm_gb300.so`` and declares its
entry points. There is no fallback: if the library is missing the import of
any compute entry point raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libmm_gb300.so")

MM_OK = 0
STATUS_NAMES = {
    0: "MM_OK", 1: "MM_ERR_INVALID_ARG", 2: "MM_ERR_UNSORTED", 3: "MM_ERR_DUPLICATE_TIME",
    4: "MM_ERR_DEGENERATE_SPAN", 5: "MM_ERR_CUTOFF", 6: "MM_ERR_OOM", 7: "MM_ERR_CUDA",
    8: "MM_ERR_TIMEOUT", 9: "MM_ERR_ZERO_VARIANCE", 10: "MM_ERR_NONFINITE", 11: "MM_ERR_UNSUPPORTED",
}
KERNELS = {"gauss": 0, "kb": 1, "es": 2}
BASES = {"dirichlet": 0, "fejer": 1}
PRECISIONS = {"fp64": 0, "bf16x3": 1, "3xtf32": 2}
SPREAD_ALGOS = {"default": 0, "scatter": 1, "gather": 2, "fused": 3}
GRAM_ALGOS = {"default": 0, "convert": 1, "tma": 2}
FFT_ALGOS = {"default": 0, "two_pass": 1, "asset": 2, "asset_pair": 4, "asset_perm": 5}
STAGES = ["prep", "spread", "fft_cols", "fft_rows", "gram", "reduce", "setup", "fused", "fft", "split"]


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int32),
        ("N_max", ctypes.c_int32),
        ("max_events", ctypes.c_int64),
        ("tol", ctypes.c_double),
        ("kernel", ctypes.c_int),
        ("basis", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("spread_tile", ctypes.c_int32),
        ("spread_algo", ctypes.c_int32),
        ("fft_algo", ctypes.c_int32),
        ("gram_algo", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("msp", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("Mr", ctypes.c_int64),
        ("fft_P", ctypes.c_int64),
        ("fft_Q", ctypes.c_int64),
        ("workspace_bytes", ctypes.c_int64),
        ("launches", ctypes.c_int64),
        ("gram_splits", ctypes.c_int32),
        ("spread_algo", ctypes.c_int32),
        ("spread_tile", ctypes.c_int32),
        ("fft_lg_cols", ctypes.c_int32),
        ("fft_rowblk", ctypes.c_int32),
        ("tuned_ms", ctypes.c_float),
        ("fft_algo", ctypes.c_int32),
        ("fft_passes", ctypes.c_int32),
        ("fft_radix", ctypes.c_int32 * 4),
        ("fft_split", ctypes.c_int32),
        ("spread_poly", ctypes.c_int32),
        ("graphs", ctypes.c_int32),
        ("graph_launches", ctypes.c_int64),
        ("gram_algo", ctypes.c_int32),
        ("res_sub", ctypes.c_int32),
    ]


class BatchDesc(ctypes.Structure):
    _fields_ = [
        ("reps", ctypes.c_int32),
        ("D", ctypes.c_int32),
        ("N_max", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("max_events", ctypes.c_int64),
        ("tol", ctypes.c_double),
        ("kernel", ctypes.c_int),
        ("basis", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("spread_algo", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 4),
    ]


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("graph_launches", ctypes.c_int64),
        ("launches", ctypes.c_int64),
        ("Mr", ctypes.c_int64),
        ("graph_captures", ctypes.c_int32),
        ("graph_kernels", ctypes.c_int32),
        ("spread_tile", ctypes.c_int32),
        ("fft_algo", ctypes.c_int32),
        ("fft_split", ctypes.c_int32),
        ("fft_passes", ctypes.c_int32),
        ("tuned_ms", ctypes.c_float),
    ]


class ServerDesc(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int32),
        ("N_max", ctypes.c_int32),
        ("max_events", ctypes.c_int64),
        ("request_max_events", ctypes.c_int64),
        ("hbm_budget", ctypes.c_int64),
        ("max_slots", ctypes.c_int32),
        ("cache_rows", ctypes.c_int32),
        ("tol", ctypes.c_double),
        ("kernel", ctypes.c_int),
        ("basis", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("reserved", ctypes.c_int32 * 4),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("t0", ctypes.c_double),
        ("t1", ctypes.c_double),
        ("n_assets", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("assets", ctypes.c_void_p),
        ("dt_equiv", ctypes.c_double),
        ("h_R", ctypes.c_void_p),
        ("h_sigma_or_null", ctypes.c_void_p),
    ]


class Completion(ctypes.Structure):
    _fields_ = [
        ("ticket", ctypes.c_int64),
        ("status", ctypes.c_int32),
        ("n_assets", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("t_submit", ctypes.c_double),
        ("t_start", ctypes.c_double),
        ("t_done", ctypes.c_double),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("slot_bytes", ctypes.c_int64),
        ("resident_bytes", ctypes.c_int64),
        ("slots", ctypes.c_int32),
        ("inflight", ctypes.c_int32),
        ("peak_inflight", ctypes.c_int32),
        ("queued", ctypes.c_int32),
        ("launches", ctypes.c_int64),
        ("cache_hits", ctypes.c_int64),
        ("cache_misses", ctypes.c_int64),
    ]


_lib = None


def load():
    """Load libmm_gb300.so (built by paper_2003_02842_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"CUDA library {LIB_PATH} is missing; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    p, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "mm_plan_create": ([ctypes.POINTER(PlanDesc), ctypes.POINTER(p)], st),
        "mm_destroy": ([p], st),
        "mm_coeffs": ([p, p, p, p, i32, d, d, p, ctypes.POINTER(i32), p], st),
        "mm_cov": ([p, p, i32, p, p], st),
        "mm_corr": ([p, p, i32, p, p, p], st),
        "mm_estimate": ([p, p, p, p, i32, d, d, p, p, p, ctypes.POINTER(i32), p], st),
        "mm_corr_noalloc": ([i32, i32, st, st, p, p, p, p], st),
        "mm_corr_pairwise": ([p, p, i32, p, i32, p, p, p, p], st),
        "mm_estimate_host": ([p, p, p, p, i32, d, d, p, p, p, ctypes.POINTER(i32), p], st),
        "mm_nyquist": ([p, p, p, d, d, ctypes.POINTER(i32), p], st),
        "mm_autotune": ([p, p, p, p, i32, d, d, p, i32, p], st),
        "mm_plan_sync": ([p], st),
        "mm_plan_get_info": ([p, ctypes.POINTER(PlanInfo)], st),
        "mm_profile_enable": ([p, i32], st),
        "mm_plan_set_graphs": ([p, i32], st),
        "mm_plan_set_wait_limit": ([p, ctypes.c_int64], st),
        "mm_profile_read": ([p, p, p, i32], st),
        "mm_status_string": ([st], ctypes.c_char_p),
        "mm_version": ([], i32),
        "mm_batch_create": ([ctypes.POINTER(BatchDesc), ctypes.POINTER(p)], st),
        "mm_batch_destroy": ([p], st),
        "mm_batch_epps": ([p, p, p, p, ctypes.POINTER(i32), i32, p, p, p], st),
        "mm_batch_autotune": ([p, p, p, p, i32, i32, p], st),
        "mm_batch_coeffs": ([p, ctypes.POINTER(p), ctypes.POINTER(i32)], st),
        "mm_batch_copy_coeffs": ([p, p, p], st),
        "mm_batch_sync": ([p], st),
        "mm_batch_profile_enable": ([p, i32], st),
        "mm_server_create": ([ctypes.POINTER(ServerDesc), ctypes.POINTER(p)], st),
        "mm_server_load": ([p, p, p, p], st),
        "mm_server_submit": ([p, ctypes.POINTER(Request), ctypes.POINTER(i64)], st),
        "mm_server_poll": ([p, ctypes.POINTER(Completion), i32, ctypes.POINTER(i32), d], st),
        "mm_server_get_stats": ([p, ctypes.POINTER(ServerStats)], st),
        "mm_server_destroy": ([p], st),
        "mm_batch_profile_read": ([p, p, p, i32], st),
        "mm_batch_get_info": ([p, ctypes.POINTER(BatchInfo)], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L
