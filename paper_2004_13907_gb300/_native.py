"""ctypes declarations of the C ABI in include/spgemm.h (argument marshalling only)."""

from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspgemm.so")

c_i32, c_i64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p

STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "INVALID_CSR", 3: "OOM", 4: "INDEX_OVERFLOW", 5: "CUDA",
    6: "TIMEOUT", 7: "REJECTED", 8: "NOT_READY", 9: "UNSUPPORTED", 10: "INTERNAL",
}
STATUS_CODES = {name: code for code, name in STATUS_NAMES.items()}
F64, F32_COMPENSATED = 0, 1


class SpgemmError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"SPGEMM_ERR_{self.name}: {message}")


class CsrIn(ctypes.Structure):
    _fields_ = [("rows", c_i64), ("cols", c_i64), ("nnz", c_i64), ("idx64_rowptr", c_i32),
                ("reserved_", c_i32), ("row_ptr", c_vp), ("col", c_vp), ("val", c_vp)]


class CsrOut(ctypes.Structure):
    _fields_ = [("rows", c_i64), ("cols", c_i64), ("nnz", c_i64), ("idx64_rowptr", c_i32),
                ("reserved_", c_i32), ("row_ptr", c_vp), ("col", c_vp), ("val", c_vp)]


ALLOC_FN = ctypes.CFUNCTYPE(c_vp, ctypes.c_size_t, c_vp, c_vp)
FREE_FN = ctypes.CFUNCTYPE(None, c_vp, c_vp, c_vp)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_vp)]


class Opts(ctypes.Structure):
    _fields_ = [("validate", c_i32), ("tiny_max", c_i32), ("warp_max", c_i32), ("block_max", c_i32),
                ("window_hash_fill", c_i32), ("force_window", c_i32), ("rowptr32_limit", c_i64),
                ("f32c_rerun_all", c_i32), ("f32c_rerun_none", c_i32), ("num_streams", c_i32),
                ("record_timings", c_i32), ("window_split_max_mb", c_i32), ("max_sms", c_i32),
                ("window_cols_max_mb", c_i32), ("fp64_accumulate", c_i32), ("general_path", c_i32),
                ("host_panels", c_i32), ("reserved", c_i32 * 8)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("rows", c_i64), ("inner", c_i64), ("cols", c_i64), ("products", c_i64),
                ("nnz_c", c_i64), ("max_row_products", c_i64), ("sym_class_rows", c_i64 * 16),
                ("num_class_rows", c_i64 * 16), ("num_class_products", c_i64 * 16),
                ("num_class_annz", c_i64 * 16), ("num_class_cnnz", c_i64 * 16), ("workspace_bytes", c_i64),
                ("f32c_rerun_rows", c_i64), ("kernel_launches", c_i64), ("needs_rowptr64", c_i32),
                ("state", c_i32)]


STAGES = ["validate", "count", "sym_window", "sym_block", "sym_warp", "sym_tiny", "sym_scan",
          "num_rowptr", "num_window", "num_block", "num_warp", "num_tiny", "num_rerun", "num_expand"]
SYM_CLASSES = ["win0", "win1", "win2", "win3", "block8192", "warp2048", "warp512", "warp128", "tiny", "micro",
               "empty"]
NUM_CLASSES = ["win0", "win1", "win2", "win3", "block8192", "block2048", "warp1024", "warp256", "warp64",
               "tiny", "micro", "empty"]


class Timings(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 16), ("launches", c_i32 * 16)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", c_i64), ("max_batch_entries", c_i64), ("max_batch_jobs", c_i32),
                ("batch_window_us", c_i32), ("num_streams", c_i32), ("start_paused", c_i32), ("prec", c_i32),
                ("reserve_sms", c_i32), ("small_products", c_i32), ("max_defer_ms", c_i32), ("host_panels", c_i32),
                ("reserved_", c_i32 * 3), ("opts", Opts)]


JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "rejected"}


class JobInfo(ctypes.Structure):
    _fields_ = [("state", c_i32), ("status", c_i32), ("batch", c_i64), ("batch_jobs", c_i64), ("rows", c_i64),
                ("cols", c_i64), ("nnz", c_i64), ("bytes", c_i64), ("needed_bytes", c_i64),
                ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("panels", c_i64), ("result_on_host", c_i64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, c_i64) for n in ("submitted", "completed", "failed", "rejected", "queued", "running", "batches",
                                     "splits", "products", "nnz_out", "bytes_in_use", "bytes_peak",
                                     "mem_cap_bytes")] + \
               [(n, ctypes.c_double) for n in ("latency_p50_ms", "latency_p99_ms", "latency_max_ms",
                                               "latency_mean_ms", "mean_batch_jobs", "elapsed_s", "jobs_per_s",
                                               "products_per_s")] + \
               [("kernel_launches", c_i64), ("reserved_", c_i64 * 7)]


TUNE_MAX_TRIALS = 32


class TuneReport(ctypes.Structure):
    _fields_ = [("trials", c_i32), ("reps", c_i32), ("default_ms", ctypes.c_double), ("best_ms", ctypes.c_double),
                ("trial_ms", ctypes.c_double * TUNE_MAX_TRIALS), ("trial_tiny_max", c_i32 * TUNE_MAX_TRIALS),
                ("trial_warp_max", c_i32 * TUNE_MAX_TRIALS), ("trial_block_max", c_i32 * TUNE_MAX_TRIALS),
                ("trial_window_fill", c_i32 * TUNE_MAX_TRIALS)]


# name -> (restype, argtypes); every symbol include/spgemm.h declares
SIGNATURES = {
    "spgemm_opts_default": (None, [ctypes.POINTER(Opts)]),
    "spgemm_plan": (c_i32, [ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), c_i32, ctypes.POINTER(Opts),
                            ctypes.POINTER(Allocator), c_vp, ctypes.POINTER(c_vp)]),
    "spgemm_symbolic": (c_i32, [c_vp, c_vp, ctypes.POINTER(c_i64), ctypes.POINTER(c_i32)]),
    "spgemm_numeric": (c_i32, [c_vp, ctypes.POINTER(CsrOut), c_vp]),
    "spgemm_plan_get_info": (c_i32, [c_vp, ctypes.POINTER(PlanInfo)]),
    "spgemm_plan_check": (c_i32, [c_vp, c_vp]),
    "spgemm_plan_destroy": (c_i32, [c_vp]),
    "spgemm_plan_get_timings": (c_i32, [c_vp, ctypes.POINTER(Timings)]),
    "spgemm_multiply_host": (c_i32, [ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), c_i32,
                                     ctypes.POINTER(Opts), ctypes.POINTER(Allocator), c_vp,
                                     ctypes.POINTER(CsrOut), c_i64, ctypes.POINTER(c_i64)]),
    "spgemm_multiply_noalloc": (c_i32, [ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(CsrOut),
                                        c_i64, ctypes.POINTER(c_i64), c_vp]),
    "spgemm_csr_transpose": (c_i32, [ctypes.POINTER(CsrIn), c_i32, ctypes.POINTER(CsrOut), ctypes.POINTER(Allocator),
                                     c_vp]),
    "spgemm_coo_to_csr": (c_i32, [c_i64, c_i64, c_i64, c_vp, c_vp, c_vp, c_i32, ctypes.POINTER(CsrOut),
                                  ctypes.POINTER(Allocator), c_vp]),
    "spgemm_batch": (c_i32, [c_i64, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), c_i32, ctypes.POINTER(Opts),
                             ctypes.POINTER(Allocator), c_vp, ctypes.POINTER(c_vp)]),
    "spgemm_batch_result": (c_i32, [c_vp, c_i64, ctypes.POINTER(CsrOut)]),
    "spgemm_batch_get_info": (c_i32, [c_vp, ctypes.POINTER(PlanInfo)]),
    "spgemm_batch_check": (c_i32, [c_vp, c_vp]),
    "spgemm_batch_replay": (c_i32, [c_vp, c_vp]),
    "spgemm_batch_destroy": (c_i32, [c_vp]),
    "spgemm_server_cfg_default": (c_i32, [ctypes.POINTER(ServerCfg)]),
    "spgemm_server_create": (c_i32, [ctypes.POINTER(ServerCfg), ctypes.POINTER(c_vp)]),
    "spgemm_server_submit": (c_i32, [c_vp, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(c_i64)]),
    "spgemm_server_poll": (c_i32, [c_vp, c_i64, ctypes.POINTER(JobInfo)]),
    "spgemm_server_wait": (c_i32, [c_vp, c_i64, ctypes.c_double, ctypes.POINTER(JobInfo)]),
    "spgemm_server_wait_any": (c_i32, [c_vp, ctypes.c_double, ctypes.POINTER(c_i64)]),
    "spgemm_server_result": (c_i32, [c_vp, c_i64, ctypes.POINTER(CsrOut)]),
    "spgemm_server_release": (c_i32, [c_vp, c_i64]),
    "spgemm_server_pause": (c_i32, [c_vp]),
    "spgemm_server_resume": (c_i32, [c_vp]),
    "spgemm_server_get_stats": (c_i32, [c_vp, ctypes.POINTER(ServerStats)]),
    "spgemm_server_reset_stats": (c_i32, [c_vp]),
    "spgemm_server_destroy": (c_i32, [c_vp]),
    "spgemm_autotune_batch": (c_i32, [c_i64, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), c_i32,
                                      ctypes.POINTER(Opts), c_i32, c_vp, ctypes.POINTER(Opts),
                                      ctypes.POINTER(TuneReport)]),
    "spgemm_last_error": (ctypes.c_char_p, []),
    "spgemm_version": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Loads libspgemm.so (built in-tree by ``build.py``). There is no fallback: without
    the library no product can be computed, and this raises."""
    global _lib
    if _lib is not None and path is None:   # loaded already (no lock on this path)
        return _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"{p} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`"
                              " (the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def check(status: int) -> None:
    if status != 0:
        msg = load().spgemm_last_error()
        raise SpgemmError(status, msg.decode() if msg else "")
