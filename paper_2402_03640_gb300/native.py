"""ctypes view of libmsat.so (the C ABI declared in include/msat.h).

Argument marshalling only: every step of the solving loop runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

MSAT_OK = 0
MSAT_EINVAL = -1
MSAT_ENOMEM = -2
MSAT_EBUDGET = -3
MSAT_ETIMEOUT = -4
MSAT_ECUDA = -5
MSAT_EAGAIN = -6
MSAT_ESTATE = -7

BACKEND_SPARSE = 0
BACKEND_DENSE = 1

_ERRNAMES = {MSAT_EINVAL: "EINVAL", MSAT_ENOMEM: "ENOMEM", MSAT_EBUDGET: "EBUDGET",
             MSAT_ETIMEOUT: "ETIMEOUT", MSAT_ECUDA: "ECUDA", MSAT_EAGAIN: "EAGAIN",
             MSAT_ESTATE: "ESTATE"}


class MsatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"msat {_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class msat_config(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("restarts", ctypes.c_int32),
                ("f_mode", ctypes.c_int32), ("seed_x", ctypes.c_uint64),
                ("heavy_deg", ctypes.c_int32), ("fwd_vw", ctypes.c_int32),
                ("stage_vw", ctypes.c_int32), ("fwd_blocks", ctypes.c_int32),
                ("light_rows", ctypes.c_int32), ("loss_norm", ctypes.c_int32),
                ("row_order", ctypes.c_int32)]


class msat_tune_entry(ctypes.Structure):
    _fields_ = [("fwd_vw", ctypes.c_int32), ("stage_vw", ctypes.c_int32),
                ("light_rows", ctypes.c_int32), ("ms_per_step", ctypes.c_float)]


F_MODES = {"auto": 0, "store": 1, "recompute": 2, "expanded": 3}
LOSS_NORMS = {"mean_unsat": 0, "sum_unsat": 1, "mean_all": 2}


class msat_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("restarts", ctypes.c_int32), ("m", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("steps_done", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("max_clause_len", ctypes.c_int32),
                ("max_degree", ctypes.c_int32), ("n_heavy", ctypes.c_int32),
                ("uniform_len", ctypes.c_int32), ("small_kernel", ctypes.c_int32)]


class msat_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_slots", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("chunk", ctypes.c_int32), ("batch_mlits", ctypes.c_int32),
                ("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


class msat_request(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_int32), ("steps", ctypes.c_int32), ("n_clauses", ctypes.c_int64),
                ("clause_off", ctypes.c_void_p), ("lits", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("seed_x", ctypes.c_uint64)]


class msat_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("best_restart", ctypes.c_int32),
                ("best_cost", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("n_vars", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("best_step", ctypes.c_int64)]


class msat_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("queued", ctypes.c_int32), ("running", ctypes.c_int32),
                ("peak_running", ctypes.c_int32), ("small_direct", ctypes.c_int32),
                ("hbm_in_use", ctypes.c_int64), ("hbm_budget", ctypes.c_int64),
                ("rounds", ctypes.c_int64), ("graph_captures", ctypes.c_int64)]


class msat_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 4), ("ms", ctypes.c_double * 4)]


STEP_NO_FINAL_EVAL = 1
STEP_GRAPH = 2
STEP_PER_PASS = 4
PROFILE_KINDS = ("forward", "backward", "evaluate", "other")

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.SO_PATH


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libmsat.so.  Raises if it is missing (build it with build.py or
    __graft_entry__.build()); build_if_missing compiles it first."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.SO_PATH
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"{path} is not built; run paper_2402_03640_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        sig = {
            "msat_config_default": ([P], ctypes.c_int),
            "msat_create": ([P, i32, i64, P, P, P, P, P], ctypes.c_int),
            "msat_destroy": ([P], None),
            "msat_set_stream": ([P, P], ctypes.c_int),
            "msat_step": ([P, i32, P, P], ctypes.c_int),
            "msat_evaluate": ([P, P, i32, P, i32], ctypes.c_int),
            "msat_best": ([P, P, P], ctypes.c_int),
            "msat_get_x": ([P, P], ctypes.c_int),
            "msat_forward": ([P, P, P, P], ctypes.c_int),
            "msat_backward": ([P, P, P], ctypes.c_int),
            "msat_get_info": ([P, P], ctypes.c_int),
            "msat_get_state": ([P, P, P, P, P, P, P, P], ctypes.c_int),
            "msat_set_state": ([P, P, P, P, P, P, i64, P], ctypes.c_int),
            "msat_step_ex": ([P, i32, ctypes.c_uint32, P, P], ctypes.c_int),
            "msat_solve": ([P, i64, ctypes.c_double, i32, P, P, P, P, i32, P], ctypes.c_int),
            "msat_autotune": ([i32, i64, P, P, P, P, P, i32, P, P, i32, P], ctypes.c_int),
            "msat_heuristic_gap": ([P, P, P], ctypes.c_int),
            "msat_selftest_bounded_wait": ([i64], ctypes.c_int),
            "msat_dense_mma_rate": ([i32, i32, P], ctypes.c_int),
            "msat_best_step": ([P, P], ctypes.c_int),
            "msat_profile_enable": ([P, ctypes.c_int], ctypes.c_int),
            "msat_profile_read": ([P, P, ctypes.c_int], ctypes.c_int),
            "msat_objective_noalloc": ([i32, i64, P, P, P, P, i32, P, P, P], ctypes.c_int),
            "msat_check": ([P], ctypes.c_int),
            "msat_evaluate_x": ([P, i32, P], ctypes.c_int),
            "msat_server_config_default": ([P], ctypes.c_int),
            "msat_server_create": ([P, P], ctypes.c_int),
            "msat_server_destroy": ([P], None),
            "msat_submit": ([P, P, P], ctypes.c_int),
            "msat_poll": ([P, ctypes.c_uint64, P, P, P], ctypes.c_int),
            "msat_wait": ([P, ctypes.c_uint64, ctypes.c_double, P, P, P], ctypes.c_int),
            "msat_cancel": ([P, ctypes.c_uint64], ctypes.c_int),
            "msat_server_get_stats": ([P, P], ctypes.c_int),
            "msat_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def check(rc: int) -> None:
    if rc != MSAT_OK:
        msg = load().msat_last_error()
        raise MsatError(rc, msg.decode() if msg else "")
