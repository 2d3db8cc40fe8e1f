"""ctypes declarations of include/ac.h and the loader of libac.so.

Argument marshalling only. There is no fallback: if the library is missing
the import of the package's compute functions raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libac.so")

# ------------------------------------------------------------------ status
AC_OK = 0
AC_ERR_INVALID_ARG = -1
AC_ERR_ALPHABET = -2
AC_ERR_EMPTY_PATTERN = -3
AC_ERR_TOO_LARGE = -4
AC_ERR_OOM = -5
AC_ERR_OVERFLOW = -6
AC_ERR_CUDA = -7
AC_ERR_TIMEOUT = -8
AC_ERR_BUSY = -9
AC_ERR_NOT_FOUND = -10
AC_ERR_NO_DEVICE = -11

AC_BUILD_FOLD_CASE = 1
AC_BUILD_HOST_ONLY = 2
AC_BUILD_NO_STRIDE2 = 4
AC_BUILD_FAILURELESS = 8
AC_BUILD_NO_STRIDE3 = 16
AC_TEXT_ASCII = 0
AC_TEXT_PACKED2 = 1
AC_SCAN_FOLD_CASE = 1
AC_NOALLOC_MAX_STATES = 1 << 21

u32, u64, i32, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64
P = ctypes.c_void_p


class BuildOpts(ctypes.Structure):
    _fields_ = [("flags", u32), ("stride2_states", u32), ("stride3_states", u32)]


class DfaInfo(ctypes.Structure):
    _fields_ = [
        ("n_states", u32), ("n_patterns", u32), ("max_len", u32), ("min_len", u32),
        ("max_depth", u32), ("on_device", u32), ("table_bytes", u64), ("out_entries", u64),
        ("device_bytes", u64), ("build_ms", ctypes.c_double), ("table2_bytes", u64), ("table3_bytes", u64),
    ]


class DfaTables(ctypes.Structure):
    _fields_ = [(k, ctypes.POINTER(u32))
                for k in ("delta", "out_off", "out_pid", "pat_len", "pat_state", "depth", "fail", "delta2", "gotos",
                          "own_off", "own_pid", "delta3")]


class Text(ctypes.Structure):
    _fields_ = [("data", P), ("n_bases", u64), ("encoding", i32), ("on_device", i32)]


class Match(ctypes.Structure):
    _fields_ = [("pos", u64), ("pattern_id", u32), ("text_id", u32)]


class Result(ctypes.Structure):
    _fields_ = [
        ("matches", P), ("capacity", u64), ("n_matches", u64), ("counts", P),
        ("on_device", i32), ("reserved", i32), ("bad_offset", u64),
    ]


class ScanOpts(ctypes.Structure):
    _fields_ = [
        ("range_begin", u64), ("range_end", u64), ("chunk", u32), ("threads", u32),
        ("interleave", u32), ("hot_states", i32), ("flags", u32), ("text_id", u32), ("stride", u32),
        ("chunks_per_lane", u32),
    ]


class ScanStats(ctypes.Structure):
    _fields_ = [
        ("total_ms", ctypes.c_float), ("scan_ms", ctypes.c_float), ("pack_ms", ctypes.c_float),
        ("counts_ms", ctypes.c_float), ("chunk", u32), ("threads", u32), ("interleave", u32),
        ("hot_states", u32), ("grid", u32), ("blocks_per_sm", u32), ("stride", u32), ("chunks_per_lane", u32),
        ("bases_walked", u64),
    ]


class ServeOpts(ctypes.Structure):
    _fields_ = [
        ("device_budget_bytes", u64), ("n_streams", u32), ("max_batch", u32), ("max_queue", u32),
        ("match_capacity_per_base_x1000", u32),
    ]


class Served(ctypes.Structure):
    _fields_ = [("matches", P), ("n_matches", u64), ("counts", P), ("n_counts", u64), ("handle", P)]


class ServeStats(ctypes.Structure):
    _fields_ = [
        ("submitted", u64), ("completed", u64), ("rejected", u64), ("failed", u64),
        ("bases_completed", u64), ("batches_launched", u64), ("p50_ms", ctypes.c_double),
        ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
        ("busy_s", ctypes.c_double), ("gbases_per_s", ctypes.c_double), ("overflow_batches", u64),
        ("cancelled", u64),
    ]


class MemUsage(ctypes.Structure):
    _fields_ = [
        ("pool_used_bytes", u64), ("pool_reserved_bytes", u64), ("live_bytes", u64), ("live_allocations", u64),
        ("allocations_seen", u64), ("launches_seen", u64),
    ]


# name -> (restype, argtypes); every function declared in include/ac.h
SIGNATURES = {
    "ac_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "ac_build": (ctypes.c_int, [P, P, u32, P, ctypes.POINTER(P)]),
    "ac_free": (None, [P]),
    "ac_dfa_info": (ctypes.c_int, [P, ctypes.POINTER(DfaInfo)]),
    "ac_dfa_tables": (ctypes.c_int, [P, ctypes.POINTER(DfaTables)]),
    "ac_pack": (ctypes.c_int, [P, u64, P, u32, ctypes.POINTER(u64), P]),
    "ac_scan": (ctypes.c_int, [P, ctypes.POINTER(Text), ctypes.POINTER(Result), ctypes.POINTER(ScanOpts), P,
                               ctypes.POINTER(ScanStats)]),
    "ac_scan_noalloc": (ctypes.c_int, [P, ctypes.POINTER(Text), ctypes.POINTER(Result), ctypes.POINTER(ScanOpts), P]),
    "ac_scan_batch": (ctypes.c_int, [P, ctypes.POINTER(Text), u32, ctypes.POINTER(Result),
                                     ctypes.POINTER(ScanOpts), P, ctypes.POINTER(ScanStats)]),
    "ac_scan_failureless": (ctypes.c_int, [P, ctypes.POINTER(Text), ctypes.POINTER(Result), ctypes.POINTER(ScanOpts), P,
                                           ctypes.POINTER(ScanStats)]),
    "ac_build_partitioned": (ctypes.c_int, [P, P, u32, u32, P, ctypes.POINTER(P)]),
    "ac_part_set_info": (ctypes.c_int, [P, ctypes.POINTER(u32), ctypes.POINTER(u32)]),
    "ac_scan_partitioned": (ctypes.c_int, [P, ctypes.POINTER(Text), ctypes.POINTER(Result), ctypes.POINTER(ScanOpts), P,
                                           ctypes.POINTER(ScanStats)]),
    "ac_part_set_free": (None, [P]),
    "ac_stream_create": (ctypes.c_int, [P, ctypes.POINTER(P)]),
    "ac_stream_scan": (ctypes.c_int, [P, ctypes.POINTER(Text), ctypes.POINTER(Result), ctypes.POINTER(ScanOpts), P,
                                      ctypes.POINTER(ScanStats)]),
    "ac_stream_reset": (ctypes.c_int, [P]),
    "ac_stream_free": (None, [P]),
    "ac_batch_plan_create": (ctypes.c_int, [P, ctypes.POINTER(Text), u32, ctypes.POINTER(Result),
                                            ctypes.POINTER(ScanOpts), P, ctypes.POINTER(P)]),
    "ac_batch_plan_run": (ctypes.c_int, [P, P, ctypes.c_int, ctypes.POINTER(Result)]),
    "ac_batch_plan_free": (None, [P]),
    "ac_autotune": (ctypes.c_int, [P, ctypes.POINTER(Text), ctypes.POINTER(ScanOpts), P]),
    "ac_autotune_batch": (ctypes.c_int, [P, ctypes.POINTER(Text), u32, ctypes.POINTER(ScanOpts), P]),
    "ac_serve_create": (ctypes.c_int, [ctypes.POINTER(ServeOpts), ctypes.POINTER(P)]),
    "ac_serve_add_dfa": (ctypes.c_int, [P, P, ctypes.POINTER(u32)]),
    "ac_serve_submit": (ctypes.c_int, [P, u32, ctypes.POINTER(Text), ctypes.POINTER(u64)]),
    "ac_serve_wait": (ctypes.c_int, [P, u64, ctypes.POINTER(Result), i64]),
    "ac_serve_take": (ctypes.c_int, [P, u64, ctypes.POINTER(Served), i64]),
    "ac_serve_release": (None, [P]),
    "ac_serve_cancel": (ctypes.c_int, [P, u64]),
    "ac_serve_stats": (ctypes.c_int, [P, ctypes.POINTER(ServeStats)]),
    "ac_serve_destroy": (None, [P]),
    "ac_fault_inject": (ctypes.c_int, [ctypes.c_char_p]),
    "ac_mem_usage": (ctypes.c_int, [ctypes.POINTER(MemUsage)]),
}

_LIB: ctypes.CDLL | None = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libac.so; raise if it has not been built (there is no fallback)."""
    global _LIB
    if _LIB is not None and path == LIB_PATH:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(
            f"libac.so not found at {path}: build it first (python -m paper_1403_7294_gb300._compile); "
            "there is no CPU fallback"
        )
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _LIB = lib
    return lib


class AcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = load().ac_status_str(status).decode()
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def check(status: int, what: str = "") -> int:
    if status != AC_OK:
        raise AcError(status, what)
    return status
