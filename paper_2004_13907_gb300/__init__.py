"""GB300 (sm_103a) sparse matrix-matrix product C = A*B on CSR matrices.

A thin Python binding of the C ABI in ``include/spgemm.h`` with the same entry-point
names. It only marshals arguments (device pointers from torch tensors, the current CUDA
stream); every step of the product runs in the library's CUDA kernels. PyTorch provides
device memory and streams.

The product is the row-by-row (Gustavson) formulation of the paper's Algorithm 1
(Sec. III-A): row i of C merges, by column, the rows of B named by row i of A scaled by
the matching entries of A, sorted by column, one entry per column that received a partial
product.
"""

from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import torch

from . import _native
from ._native import F32_COMPENSATED, F64, SpgemmError  # noqa: F401

__all__ = [
    "DeviceCSR", "Plan", "SpgemmError", "F64", "F32_COMPENSATED", "spgemm_opts_default",
    "spgemm_plan", "spgemm_symbolic", "spgemm_numeric", "spgemm_plan_get_info",
    "spgemm_plan_check", "spgemm_plan_get_timings", "spgemm_plan_destroy", "spgemm_multiply_host", "spgemm_multiply_noalloc",
    "spgemm_last_error", "spgemm_version", "multiply", "lib", "Batch", "spgemm_batch", "Server",
    "spgemm_server_cfg_default", "spgemm_autotune_batch", "csr_transpose", "coo_to_csr", "multiply_csc",
]


def lib() -> ctypes.CDLL:
    return _native.load()


def _prec(p) -> int:
    if p is F64 or p is F32_COMPENSATED:
        return p
    if p in (F64, "f64", "fp64", torch.float64):
        return F64
    if p in (F32_COMPENSATED, "f32c", "fp32c", "f32", torch.float32):
        return F32_COMPENSATED
    raise ValueError(f"unknown precision {p!r}")


def _vdtype(prec: int) -> torch.dtype:
    return torch.float64 if prec == F64 else torch.float32


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream_handle(stream) -> int:
    if stream is None:
        if _raw_stream is not None:
            return _raw_stream(torch._C._cuda_getDevice())
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


@dataclass
class DeviceCSR:
    """A CSR matrix whose arrays are torch tensors (device, or host for the host entry)."""

    rows: int
    cols: int
    row_ptr: torch.Tensor   # int32 or int64, rows+1
    col: torch.Tensor       # int32, nnz
    val: torch.Tensor       # float64 or float32, nnz

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def idx64(self) -> int:
        return 1 if self.row_ptr.dtype == torch.int64 else 0

    @staticmethod
    def from_host(M, device="cuda", dtype=None, idx64: bool = False) -> "DeviceCSR":
        """From a host CSR (numpy arrays ``row_ptr``, ``col``, ``val``)."""
        rp = torch.as_tensor(M.row_ptr).to(torch.int64 if idx64 else torch.int32)
        col = torch.as_tensor(M.col).to(torch.int32)
        val = torch.as_tensor(M.val)
        if dtype is not None:
            val = val.to(dtype)
        return DeviceCSR(int(M.rows), int(M.cols), rp.to(device), col.to(device), val.to(device))

    def to_host(self):
        return DeviceCSR(self.rows, self.cols, self.row_ptr.cpu(), self.col.cpu(), self.val.cpu())

    def as_in(self) -> _native.CsrIn:
        return _native.CsrIn(self.rows, self.cols, self.nnz, self.idx64, 0, self.row_ptr.data_ptr(),
                             self.col.data_ptr(), self.val.data_ptr())

    def as_out(self) -> _native.CsrOut:
        return _native.CsrOut(self.rows, self.cols, self.nnz, self.idx64, 0, self.row_ptr.data_ptr(),
                              self.col.data_ptr(), self.val.data_ptr())


class Plan:
    """Handle of a native plan; keeps the input tensors alive while the plan holds their
    pointers."""

    def __init__(self, handle: int, A: DeviceCSR, B: DeviceCSR, prec: int):
        self.handle = handle
        self.A, self.B, self.prec = A, B, prec
        self.nnz_c = -1
        self.needs_rowptr64 = 0

    def __del__(self):
        try:
            if self.handle:
                lib().spgemm_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def spgemm_opts_default(**overrides) -> _native.Opts:
    o = _native.Opts()
    lib().spgemm_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(f"spgemm_opts has no field {k}")
        setattr(o, k, v)
    return o


def spgemm_plan(A: DeviceCSR, B: DeviceCSR, prec=F64, opts: _native.Opts | None = None,
                stream=None) -> Plan:
    prec = _prec(prec)
    a, b = A.as_in(), B.as_in()
    h = ctypes.c_void_p()
    st = lib().spgemm_plan(ctypes.byref(a), ctypes.byref(b), prec,
                           ctypes.byref(opts) if opts is not None else None, None,
                           _stream_handle(stream), ctypes.byref(h))
    _native.check(st)
    return Plan(h.value, A, B, prec)


def spgemm_symbolic(plan: Plan, stream=None) -> tuple:
    nnz = ctypes.c_int64()
    need = ctypes.c_int32()
    _native.check(lib().spgemm_symbolic(plan.handle, _stream_handle(stream), ctypes.byref(nnz),
                                        ctypes.byref(need)))
    plan.nnz_c, plan.needs_rowptr64 = int(nnz.value), int(need.value)
    return plan.nnz_c, plan.needs_rowptr64


def spgemm_numeric(plan: Plan, C: DeviceCSR, stream=None) -> DeviceCSR:
    c = C.as_out()
    _native.check(lib().spgemm_numeric(plan.handle, ctypes.byref(c), _stream_handle(stream)))
    return C


def spgemm_plan_get_info(plan: Plan) -> dict:
    info = _native.PlanInfo()
    _native.check(lib().spgemm_plan_get_info(plan.handle, ctypes.byref(info)))
    out = {}
    for name, _ in _native.PlanInfo._fields_:
        v = getattr(info, name)
        out[name] = list(v) if not isinstance(v, int) else v
    return out


def spgemm_plan_get_timings(plan: Plan) -> dict:
    """Per-stage device milliseconds and launch counts of the last run of each stage
    (needs ``record_timings=1`` in the plan's options)."""
    t = _native.Timings()
    _native.check(lib().spgemm_plan_get_timings(plan.handle, ctypes.byref(t)))
    return {name: (t.ms[i], t.launches[i]) for i, name in enumerate(_native.STAGES)}


def spgemm_plan_check(plan: Plan, stream=None) -> None:
    _native.check(lib().spgemm_plan_check(plan.handle, _stream_handle(stream)))


def spgemm_plan_destroy(plan: Plan) -> None:
    if plan.handle:
        _native.check(lib().spgemm_plan_destroy(plan.handle))
        plan.handle = None


def spgemm_last_error() -> str:
    return lib().spgemm_last_error().decode()


def spgemm_version() -> str:
    return lib().spgemm_version().decode()


def alloc_output(plan: Plan, idx64: bool | None = None, device=None) -> DeviceCSR:
    """Allocates C for a plan after spgemm_symbolic (row_ptr int64 when required)."""
    if plan.nnz_c < 0:
        raise RuntimeError("spgemm_symbolic has not run")
    dev = device if device is not None else plan.A.col.device
    use64 = plan.needs_rowptr64 if idx64 is None else int(idx64)
    rp = torch.empty(plan.A.rows + 1, dtype=torch.int64 if use64 else torch.int32, device=dev)
    col = torch.empty(plan.nnz_c, dtype=torch.int32, device=dev)
    val = torch.empty(plan.nnz_c, dtype=_vdtype(plan.prec), device=dev)
    return DeviceCSR(plan.A.rows, plan.B.cols, rp, col, val)


def multiply(A: DeviceCSR, B: DeviceCSR, prec=F64, opts: _native.Opts | None = None, stream=None,
             idx64: bool | None = None, check: bool = False) -> DeviceCSR:
    """C = A*B on the device: plan, symbolic, allocate C, numeric (asynchronous after the
    symbolic pass's read-back of nnz(C))."""
    plan = spgemm_plan(A, B, prec, opts, stream)
    spgemm_symbolic(plan, stream)
    C = alloc_output(plan, idx64)
    spgemm_numeric(plan, C, stream)
    if check:
        spgemm_plan_check(plan, stream)
    spgemm_plan_destroy(plan)
    return C


class _DevArray:
    """__cuda_array_interface__ over library-owned device memory (no copy)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def _view(ptr: int, n: int, dtype: torch.dtype, device) -> torch.Tensor:
    if n == 0:
        return torch.empty(0, dtype=dtype, device=device)
    typestr = {torch.int32: "<i4", torch.int64: "<i8", torch.float64: "<f8", torch.float32: "<f4"}[dtype]
    return torch.as_tensor(_DevArray(ptr, n, typestr), device=device)


class Batch:
    """Handle of a native batch (stacked block-diagonal product). The result tensors returned by
    ``result`` are views of memory the batch owns: keep the Batch alive while using them."""

    def __init__(self, handle: int, As, Bs, prec: int):
        self.handle = handle
        self.As, self.Bs, self.prec = As, Bs, prec
        self.device = As[0].col.device if As else torch.device("cuda")

    def __len__(self):
        return len(self.As)

    def result(self, j: int) -> DeviceCSR:
        c = _native.CsrOut()
        _native.check(lib().spgemm_batch_result(self.handle, j, ctypes.byref(c)))
        vdt = _vdtype(self.prec)
        return DeviceCSR(int(c.rows), int(c.cols), _view(c.row_ptr, c.rows + 1, torch.int64, self.device),
                         _view(c.col, c.nnz, torch.int32, self.device), _view(c.val, c.nnz, vdt, self.device))

    def info(self) -> dict:
        info = _native.PlanInfo()
        _native.check(lib().spgemm_batch_get_info(self.handle, ctypes.byref(info)))
        return {name: (list(getattr(info, name)) if not isinstance(getattr(info, name), int) else getattr(info, name))
                for name, _ in _native.PlanInfo._fields_}

    def check(self, stream=None) -> None:
        _native.check(lib().spgemm_batch_check(self.handle, _stream_handle(stream)))

    def replay(self, stream=None) -> None:
        _native.check(lib().spgemm_batch_replay(self.handle, _stream_handle(stream)))

    def destroy(self) -> None:
        if self.handle:
            _native.check(lib().spgemm_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            if self.handle:
                lib().spgemm_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def spgemm_batch(As, Bs, prec=F64, opts: _native.Opts | None = None, stream=None) -> Batch:
    """C_j = A_j * B_j for every job, computed as one stacked product (see include/spgemm.h)."""
    prec = _prec(prec)
    n = len(As)
    if n != len(Bs):
        raise ValueError("As and Bs differ in length")
    arr_a = (_native.CsrIn * n)(*[A.as_in() for A in As])
    arr_b = (_native.CsrIn * n)(*[B.as_in() for B in Bs])
    h = ctypes.c_void_p()
    _native.check(lib().spgemm_batch(n, arr_a, arr_b, prec, ctypes.byref(opts) if opts is not None else None, None,
                                     _stream_handle(stream), ctypes.byref(h)))
    return Batch(h.value, list(As), list(Bs), prec)


def spgemm_autotune_batch(As, Bs, prec=F64, base: _native.Opts | None = None, reps: int = 2,
                          stream=None) -> tuple:
    """Row-class thresholds and window merge cap for this batch, chosen by timing it (see
    include/spgemm.h). Returns (options, report) with the report's trials as a list of dicts."""
    prec = _prec(prec)
    n = len(As)
    if n != len(Bs):
        raise ValueError("As and Bs differ in length")
    arr_a = (_native.CsrIn * n)(*[A.as_in() for A in As])
    arr_b = (_native.CsrIn * n)(*[B.as_in() for B in Bs])
    best = _native.Opts()
    rep = _native.TuneReport()
    _native.check(lib().spgemm_autotune_batch(n, arr_a, arr_b, prec, ctypes.byref(base) if base is not None else None,
                                              reps, _stream_handle(stream), ctypes.byref(best), ctypes.byref(rep)))
    k = min(rep.trials, _native.TUNE_MAX_TRIALS)
    trials = [{"ms": rep.trial_ms[t], "tiny_max": rep.trial_tiny_max[t], "warp_max": rep.trial_warp_max[t],
               "block_max": rep.trial_block_max[t], "window_hash_fill": rep.trial_window_fill[t]} for t in range(k)]
    return best, {"trials": trials, "default_ms": rep.default_ms, "best_ms": rep.best_ms, "reps": rep.reps}


def spgemm_multiply_noalloc(A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, stream=None) -> int:
    """C = A*B into the caller's device arrays without any device allocation (small
    products: A.rows <= 65536, rows of C <= 4096 entries, FP64). ``C.col``/``C.val`` give the
    capacity. Returns nnz(C); raises SpgemmError (INVALID_ARG with ``nnz_c`` attached) when C
    is too small."""
    a, b, c = A.as_in(), B.as_in(), C.as_out()
    nnz = ctypes.c_int64()
    cap = min(C.col.numel(), C.val.numel())   # the kernels write both arrays up to the capacity
    st = lib().spgemm_multiply_noalloc(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), cap,
                                       ctypes.byref(nnz), _stream_handle(stream))
    if st != 0:
        msg = lib().spgemm_last_error()
        err = SpgemmError(st, msg.decode() if msg else "")
        err.nnz_c = int(nnz.value)
        raise err
    return int(nnz.value)


def csr_transpose(M: DeviceCSR, stream=None, idx64: bool | None = None) -> DeviceCSR:
    """M^T in CSR (the CSC arrays of M), converted on the device (spgemm_csr_transpose)."""
    vb = 4 if M.val.dtype == torch.float32 else 8
    if idx64 is None:
        idx64 = M.nnz > 0x7FFFFFFF
    T = DeviceCSR(M.cols, M.rows, torch.empty(M.cols + 1, dtype=torch.int64 if idx64 else torch.int32,
                                              device=M.col.device),
                  torch.empty(M.nnz, dtype=torch.int32, device=M.col.device),
                  torch.empty(M.nnz, dtype=M.val.dtype, device=M.col.device))
    a, t = M.as_in(), T.as_out()
    _native.check(lib().spgemm_csr_transpose(ctypes.byref(a), vb, ctypes.byref(t), None, _stream_handle(stream)))
    return T


def coo_to_csr(rows: int, cols: int, row: torch.Tensor, col: torch.Tensor, val: torch.Tensor, stream=None,
               idx64: bool | None = None) -> DeviceCSR:
    """Canonical CSR (columns sorted within each row) from device COO triples in any order
    (spgemm_coo_to_csr); a repeated (row, col) pair raises INVALID_CSR."""
    nnz = int(row.numel())
    if int(col.numel()) != nnz or int(val.numel()) != nnz:
        raise ValueError("row, col and val differ in length")
    row = row.to(torch.int32).contiguous()
    col = col.to(torch.int32).contiguous()
    val = val.contiguous()
    vb = 4 if val.dtype == torch.float32 else 8
    if idx64 is None:
        idx64 = nnz > 0x7FFFFFFF
    C = DeviceCSR(rows, cols, torch.empty(rows + 1, dtype=torch.int64 if idx64 else torch.int32, device=val.device),
                  torch.empty(nnz, dtype=torch.int32, device=val.device), torch.empty(nnz, dtype=val.dtype,
                                                                                     device=val.device))
    c = C.as_out()
    _native.check(lib().spgemm_coo_to_csr(rows, cols, nnz, row.data_ptr(), col.data_ptr(), val.data_ptr(), vb,
                                          ctypes.byref(c), None, _stream_handle(stream)))
    return C


def multiply_csc(A_csc: DeviceCSR, B_csc: DeviceCSR, prec=F64, opts: _native.Opts | None = None,
                 stream=None) -> DeviceCSR:
    """C = A*B for matrices held in CSC. Each argument is the CSR view of the matrix's
    transpose (its CSC arrays: column pointers, row indices, values); the result is the CSR view
    of C^T, i.e. C in CSC. No conversion runs: C^T = B^T * A^T is a CSR product of the views."""
    return multiply(B_csc, A_csc, prec, opts, stream)


def spgemm_multiply_host(A, B, prec=F64, opts: _native.Opts | None = None, stream=None,
                         out: DeviceCSR | None = None, idx64: bool = False) -> DeviceCSR:
    """C = A*B through host buffers (``DeviceCSR`` with CPU tensors, pinned for speed).
    ``out`` may hold pre-allocated host arrays (capacity = its col length); they are grown
    when nnz(C) does not fit."""
    prec = _prec(prec)
    a, b = A.as_in(), B.as_in()
    for _ in range(2):
        if out is None:
            out = DeviceCSR(A.rows, B.cols,
                            torch.empty(A.rows + 1, dtype=torch.int64 if idx64 else torch.int32),
                            torch.empty(0, dtype=torch.int32), torch.empty(0, dtype=_vdtype(prec)))
        c = out.as_out()
        cap = out.col.numel()
        nnz = ctypes.c_int64()
        st = lib().spgemm_multiply_host(ctypes.byref(a), ctypes.byref(b), prec,
                                        ctypes.byref(opts) if opts is not None else None, None,
                                        _stream_handle(stream), ctypes.byref(c), cap, ctypes.byref(nnz))
        if st == 1 and nnz.value > cap:
            pin = out.row_ptr.is_pinned()
            out = DeviceCSR(A.rows, B.cols, out.row_ptr,
                            torch.empty(nnz.value, dtype=torch.int32, pin_memory=pin),
                            torch.empty(nnz.value, dtype=_vdtype(prec), pin_memory=pin))
            continue
        _native.check(st)
        n = int(nnz.value)
        return DeviceCSR(A.rows, B.cols, out.row_ptr, out.col[:n], out.val[:n])
    raise RuntimeError("spgemm_multiply_host: capacity retry failed")


def spgemm_server_cfg_default(**overrides) -> _native.ServerCfg:
    """Server configuration with the library defaults, then ``overrides`` (field=value; ``opts``
    takes an ``Opts``, ``prec`` a precision name or code)."""
    cfg = _native.ServerCfg()
    _native.check(lib().spgemm_server_cfg_default(ctypes.byref(cfg)))
    for k, v in overrides.items():
        if k == "prec":
            v = _prec(v)
        if not hasattr(cfg, k):
            raise AttributeError(f"spgemm_server_cfg has no field {k!r}")
        setattr(cfg, k, v)
    return cfg


def _job_dict(info: _native.JobInfo) -> dict:
    d = {name: getattr(info, name) for name, _ in _native.JobInfo._fields_}
    d["state"] = _native.JOB_STATES.get(info.state, str(info.state))
    d["status"] = _native.STATUS_NAMES.get(info.status, str(info.status))
    return d


class Server:
    """Handle of a native server (continuous batching, see include/spgemm.h). The Python object
    keeps each job's input tensors alive until the job is released."""

    def __init__(self, cfg: _native.ServerCfg | None = None, **overrides):
        if cfg is None:
            cfg = spgemm_server_cfg_default(**overrides)
        self.prec = int(cfg.prec)
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        _native.check(lib().spgemm_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self._inputs = {}
        # a job may finish, and another thread release it, before submit has recorded its inputs
        self._inputs_lock = threading.Lock()

    def submit(self, A: DeviceCSR, B: DeviceCSR, sync: bool = True) -> int:
        """Queues C = A*B. The server reads A and B on its own streams, so they must be written
        before this call: with ``sync`` the current stream is synchronized first."""
        if sync:
            torch.cuda.current_stream().synchronize()
        a, b = A.as_in(), B.as_in()
        job = ctypes.c_int64()
        with self._inputs_lock:
            _native.check(lib().spgemm_server_submit(self.handle, ctypes.byref(a), ctypes.byref(b),
                                                     ctypes.byref(job)))
            self._inputs[job.value] = (A, B)
        return int(job.value)

    def poll(self, job: int) -> dict:
        """The job's state and timings; never raises for a failed job (see ``state``)."""
        info = _native.JobInfo()
        st = lib().spgemm_server_poll(self.handle, job, ctypes.byref(info))
        if st == 1:
            _native.check(st)
        return _job_dict(info)

    def wait(self, job: int, timeout: float | None = None) -> dict:
        """Waits for a final state; raises SpgemmError (TIMEOUT, or the job's own error)."""
        info = _native.JobInfo()
        _native.check(lib().spgemm_server_wait(self.handle, job, -1.0 if timeout is None else float(timeout),
                                               ctypes.byref(info)))
        return _job_dict(info)

    def wait_any(self, timeout: float | None = None) -> int | None:
        """Id of a job that reached a final state and was not returned by this call before (in the
        order they finished), waiting up to ``timeout`` seconds (None: no limit); None on timeout."""
        job = ctypes.c_int64()
        st = lib().spgemm_server_wait_any(self.handle, -1.0 if timeout is None else float(timeout),
                                          ctypes.byref(job))
        if st == _native.STATUS_CODES["TIMEOUT"]:
            return None
        _native.check(st)
        return int(job.value)

    def result(self, job: int) -> DeviceCSR:
        """View of a done job's result (valid until ``release``): device tensors, or CPU tensors over
        pinned host memory for a job the server ran as row panels (over its memory cap)."""
        info = self.poll(job)
        c = _native.CsrOut()
        _native.check(lib().spgemm_server_result(self.handle, job, ctypes.byref(c)))
        vdt = _vdtype(self.prec)
        if info["result_on_host"]:
            import numpy as np

            def host(ptr, n, ctype):
                if n == 0:
                    return torch.empty(0, dtype={ctypes.c_int64: torch.int64, ctypes.c_int32: torch.int32,
                                                 ctypes.c_double: torch.float64, ctypes.c_float: torch.float32}[ctype])
                return torch.from_numpy(np.ctypeslib.as_array((ctype * n).from_address(ptr)))
            vct = ctypes.c_double if self.prec == F64 else ctypes.c_float
            return DeviceCSR(int(c.rows), int(c.cols), host(c.row_ptr, c.rows + 1, ctypes.c_int64),
                             host(c.col, c.nnz, ctypes.c_int32), host(c.val, c.nnz, vct))
        return DeviceCSR(int(c.rows), int(c.cols), _view(c.row_ptr, c.rows + 1, torch.int64, self.device),
                         _view(c.col, c.nnz, torch.int32, self.device), _view(c.val, c.nnz, vdt, self.device))

    def release(self, job: int) -> None:
        with self._inputs_lock:
            _native.check(lib().spgemm_server_release(self.handle, job))
            self._inputs.pop(job, None)

    def pause(self) -> None:
        _native.check(lib().spgemm_server_pause(self.handle))

    def resume(self) -> None:
        _native.check(lib().spgemm_server_resume(self.handle))

    def stats(self) -> dict:
        s = _native.ServerStats()
        _native.check(lib().spgemm_server_get_stats(self.handle, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in _native.ServerStats._fields_ if name != "reserved_"}

    def reset_stats(self) -> None:
        _native.check(lib().spgemm_server_reset_stats(self.handle))

    def close(self) -> None:
        if self.handle:
            _native.check(lib().spgemm_server_destroy(self.handle))
            self.handle = None
            self._inputs.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
