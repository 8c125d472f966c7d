"""CPU oracle for C = A*B (CSR in, CSR out): TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The CUDA library never calls it and shares no code with it.

``spgemm`` is the paper's row-by-row formulation (Algorithm 1, Sec. III-A) as a plain
ordered-map Gustavson product in FP64 (``gustavson.cpp``), threaded over rows (by default with
a dense accumulator per thread instead of the map for the stored-order sums: the same additions
in the same order, bit-identical values, several times faster on wide rows). With
``exact_sum=True`` every value is instead the sum of the entry's rounded partial products
rounded once (correctly rounded, ties to even), kept exactly as Shewchuk's non-overlapping
partial sums until the end.
``products_per_row`` is the definition of the per-row intermediate-product count used by
the method's flop metric: P_i = sum over stored (i, k) of A of nnz(row k of B), the number
of partial products Algorithm 1 forms for row i (its B rows "streamed" for row i, Sec. III-A).

Parity status of each function (what pins it to something other than itself) is listed
in the test module ``tests/test_oracle_pins.py``; none is unpinned.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "gustavson.cpp")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no contraction of multiply-add)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_spgemm.restype = P
            lib.oracle_spgemm.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, ctypes.c_int64,
                                          ctypes.c_int]
            lib.oracle_spgemm_ex.restype = P
            lib.oracle_spgemm_ex.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64]
            lib.oracle_nnz.restype = ctypes.c_int64
            lib.oracle_nnz.argtypes = [P]
            lib.oracle_threads.restype = ctypes.c_int
            lib.oracle_threads.argtypes = [P]
            lib.oracle_copy.restype = None
            lib.oracle_copy.argtypes = [P, P, P, P, P, P]
            lib.oracle_free.restype = None
            lib.oracle_free.argtypes = [P]
            _lib = lib
    return _lib


@dataclass
class OracleOut:
    """Rows of C (CSR over the requested rows) with per-entry mag = sum|a*b| and term counts."""

    row_ptr: np.ndarray   # int64, len(rows)+1
    col: np.ndarray       # int32
    val: np.ndarray       # float64
    mag: np.ndarray       # float64
    terms: np.ndarray     # int32
    threads: int

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# widest C for which the dense accumulator is used (slots per thread: 20 bytes each)
DENSE_MAX_COLS = 1 << 25


def spgemm(A, B, rows=None, threads: int = 0, values: bool = True, exact_sum: bool = False,
           method: str = "auto") -> OracleOut:
    """C = A*B for the given rows of A (all rows when ``rows`` is None).

    A and B are ``synth.CSR``-like objects (rows, cols, row_ptr, col, val). Values are
    taken in FP64 (FP32 inputs are widened exactly). ``values=False`` multiplies the
    patterns (every stored value taken as 1). ``exact_sum=True`` rounds each entry's sum of
    rounded products once instead of summing in stored order. ``method``: "map" (ordered map per
    row), "dense" (dense accumulator per thread) or "auto" (dense when C has at most
    DENSE_MAX_COLS columns); both give the same values.
    """
    if method not in ("auto", "map", "dense"):
        raise ValueError(f"unknown method {method!r}")
    dense = method == "dense" or (method == "auto" and B.cols <= DENSE_MAX_COLS)
    if A.cols != B.rows:
        raise ValueError("inner dimensions differ")
    lib = _load()
    a_rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    b_rp = np.ascontiguousarray(B.row_ptr, dtype=np.int64)
    a_col = np.ascontiguousarray(A.col, dtype=np.int32)
    b_col = np.ascontiguousarray(B.col, dtype=np.int32)
    a_val = np.ascontiguousarray(A.val, dtype=np.float64) if values else None
    b_val = np.ascontiguousarray(B.val, dtype=np.float64) if values else None
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nrows = A.rows if r is None else r.shape[0]
    h = lib.oracle_spgemm_ex(A.rows, _ptr(a_rp), _ptr(a_col), _ptr(a_val), _ptr(b_rp), _ptr(b_col),
                             _ptr(b_val), _ptr(r), nrows, threads, 1 if exact_sum else 0, 1 if dense else 0,
                             int(B.cols))
    try:
        nnz = lib.oracle_nnz(h)
        rp = np.empty(nrows + 1, dtype=np.int64)
        col = np.empty(nnz, dtype=np.int32)
        val = np.empty(nnz, dtype=np.float64)
        mag = np.empty(nnz, dtype=np.float64)
        terms = np.empty(nnz, dtype=np.int32)
        lib.oracle_copy(h, _ptr(rp), _ptr(col), _ptr(val), _ptr(mag), _ptr(terms))
        nt = lib.oracle_threads(h)
    finally:
        lib.oracle_free(h)
    return OracleOut(rp, col, val, mag, terms, nt)


def products_per_row(A, B) -> np.ndarray:
    """P_i = sum over the stored columns k of row i of A of nnz(row k of B) (int64)."""
    lenB = np.diff(np.asarray(B.row_ptr, dtype=np.int64))
    lenA = np.diff(np.asarray(A.row_ptr, dtype=np.int64))
    per_entry = lenB[np.asarray(A.col, dtype=np.int64)]
    rows = np.repeat(np.arange(A.rows, dtype=np.int64), lenA)
    return np.bincount(rows, weights=per_entry, minlength=A.rows).astype(np.int64) if A.rows else \
        np.zeros(0, np.int64)
