"""ctypes declarations of the liblabs C ABI (include/labs.h).

Argument marshalling only: every computation runs in liblabs.so.  Loading fails
loudly when the library cannot be built or loaded -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

LABS_OK = 0
LABS_EINVAL = -1
LABS_ENOMEM = -2
LABS_ECUDA = -3
LABS_ETIMEOUT = -4
LABS_ECANCELLED = -5
LABS_ESTATE = -6
LABS_ERANGE = -7
LABS_ETABU_FULL = -8
LABS_MAX_L = 511
LABS_MAX_L_LONG = 11263
LABS_MAX_GROUPS = 64
LABS_TRACE_RESTART = 0x10000
LABS_TRACE_BLOCKED = -1
LABS_FLAG_NO_GRAPH = 1
LABS_FLAG_CHECK_STATE = 2
LABS_FLAG_LEARNED = 4
LABS_FLAG_WARP_PER_WALKER = 8
LABS_FLAG_TWO_PER_WARP = 16
LABS_FLAG_BEST_FIRST = 32
LABS_FLAG_PSL = 64
LABS_FLAG_SECOND_HASH = 128
LABS_FLAG_STRICT_HT = 256
LABS_FLAG_LEARNED_RESTARTS = 512
LABS_QUEUE_SIZE = 32
LABS_BEST_FIRST_MAX_STEPS = 1 << 28
LABS_BEST_FIRST_MAX_STEPS_LONG = 1 << 21
LOG_RECORD_BYTES = 64

ERRORS = {LABS_EINVAL: "EINVAL", LABS_ENOMEM: "ENOMEM", LABS_ECUDA: "ECUDA", LABS_ETIMEOUT: "ETIMEOUT",
          LABS_ECANCELLED: "ECANCELLED", LABS_ESTATE: "ESTATE", LABS_ERANGE: "ERANGE",
          LABS_ETABU_FULL: "ETABU_FULL"}

# Every exported symbol of include/labs.h, in declaration order.
EXPORTS = [
    "labs_default_config", "labs_init", "labs_init_multi", "labs_workspace_bytes", "labs_bind_workspace",
    "labs_reset", "labs_isl", "labs_neighbor_delta", "labs_walk", "labs_sync", "labs_best",
    "labs_best_psl", "labs_walker_psl", "labs_walker_results", "labs_stats", "labs_trace", "labs_enumerate_scratch_bytes", "labs_enumerate",
    "labs_enumerate_noalloc", "labs_net_sizes", "labs_net_init", "labs_net_forward", "labs_net_gradients",
    "labs_net_adamw", "labs_log", "labs_log_labels", "labs_features", "labs_learned_workspace_bytes",
    "labs_learned", "labs_trace_learned", "labs_checkpoint", "labs_restore", "labs_set_deadline", "labs_cancel", "labs_clear_stop",
    "labs_last_error", "labs_destroy",
]


class LabsConfig(ctypes.Structure):
    _fields_ = [("tabu_log2", ctypes.c_int32), ("probe_cap", ctypes.c_int32), ("patience", ctypes.c_int32),
                ("target_num", ctypes.c_int32), ("target_den", ctypes.c_int32), ("chunk_steps", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("flags", ctypes.c_int32)]


class LabsCounters(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("flip_evaluations", ctypes.c_int64), ("restarts", ctypes.c_int64),
                ("overflows", ctypes.c_int64), ("blocked", ctypes.c_int64), ("best_isl", ctypes.c_int32),
                ("best_L", ctypes.c_int32), ("best_walker", ctypes.c_int64), ("target_step", ctypes.c_int64),
                ("walkers_at_target", ctypes.c_int64), ("walkers_per_warp", ctypes.c_int32),
                ("lane_block", ctypes.c_int32), ("best_psl", ctypes.c_int32), ("tensor_cores", ctypes.c_int32),
                ("cache_hits", ctypes.c_int64)]


class LabsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Loads liblabs.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        override = os.environ.get("LABS_LIBRARY")
        if override:
            path = override  # a separately built variant of the same sources
        elif build_if_needed:
            path = _build.build()
        else:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError("liblabs.so is not built: run paper_2011_00068_gb300.build.build()")
        L = ctypes.CDLL(path)
        P, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
        pp = ctypes.POINTER(ctypes.c_void_p)
        cfgp = ctypes.POINTER(LabsConfig)
        sig = {
            "labs_default_config": (None, [cfgp]),
            "labs_init": (ctypes.c_int, [pp, i32, i64, u64, cfgp, P]),
            "labs_init_multi": (ctypes.c_int, [pp, P, P, i32, u64, cfgp, P]),
            "labs_workspace_bytes": (ctypes.c_int, [P, ctypes.POINTER(sz)]),
            "labs_bind_workspace": (ctypes.c_int, [P, P, sz]),
            "labs_reset": (ctypes.c_int, [P]),
            "labs_isl": (ctypes.c_int, [P, P, i64, P]),
            "labs_neighbor_delta": (ctypes.c_int, [P, P, i64, P]),
            "labs_walk": (ctypes.c_int, [P, i64]),
            "labs_sync": (ctypes.c_int, [P]),
            "labs_best": (ctypes.c_int, [P, i32, P, P, P, P, ctypes.c_char_p]),
            "labs_best_psl": (ctypes.c_int, [P, i32, P, P, P, P, ctypes.c_char_p]),
            "labs_walker_psl": (ctypes.c_int, [P, i64, i64, P, P]),
            "labs_walker_results": (ctypes.c_int, [P, i64, i64, P, P, P, P, P]),
            "labs_stats": (ctypes.c_int, [P, i32, ctypes.POINTER(LabsCounters)]),
            "labs_trace": (ctypes.c_int, [P, P, i32, i64, P, P]),
            "labs_enumerate_scratch_bytes": (ctypes.c_int, [i32, ctypes.POINTER(sz)]),
            "labs_enumerate": (ctypes.c_int, [i32, P, sz, P, P, P, P]),
            "labs_enumerate_noalloc": (ctypes.c_int, [i32, P, P, P, P]),
            "labs_net_sizes": (ctypes.c_int, [i32, i64, ctypes.POINTER(sz), ctypes.POINTER(sz)]),
            "labs_net_init": (ctypes.c_int, [P, u64, P]),
            "labs_net_forward": (ctypes.c_int, [P, P, i64, i32, P, P, P, sz, P]),
            "labs_net_gradients": (ctypes.c_int, [P, P, P, P, P, i64, i32, P, P, P, sz, P]),
            "labs_net_adamw": (ctypes.c_int, [P, P, P, P, i64, ctypes.c_float, ctypes.c_float, P]),
            "labs_log": (ctypes.c_int, [P, P, i64]),
            "labs_log_labels": (ctypes.c_int, [P, i64, P, P, P, P]),
            "labs_features": (ctypes.c_int, [i32, P, i64, i64, P, P]),
            "labs_learned_workspace_bytes": (ctypes.c_int, [P, i32, ctypes.POINTER(sz)]),
            "labs_learned": (ctypes.c_int, [P, P, i32, i32, P, sz]),
            "labs_trace_learned": (ctypes.c_int, [P, i32, P, P, P, P, P, P]),
            "labs_checkpoint": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.POINTER(sz)]),
            "labs_restore": (ctypes.c_int, [P, P, sz]),
            "labs_set_deadline": (ctypes.c_int, [P, u64]),
            "labs_cancel": (ctypes.c_int, [P]),
            "labs_clear_stop": (ctypes.c_int, [P]),
            "labs_last_error": (ctypes.c_char_p, [P]),
            "labs_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return _lib
