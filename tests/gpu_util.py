"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and compare it with
the CPU oracle (structure bit-exact; FP64 values within 1e-12 * sum|a*b| per entry)."""

import numpy as np
import pytest
import torch

import oracle

TOL_F64 = 1e-12


def gpu_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def run_gpu(A, B, opts=None, idx64_in=False, idx64_out=None, prec="f64", check=True):
    import paper_2004_13907_gb300 as sp
    dt = torch.float64 if prec == "f64" else torch.float32
    dA = sp.DeviceCSR.from_host(A, "cuda", dtype=dt, idx64=idx64_in)
    dB = sp.DeviceCSR.from_host(B, "cuda", dtype=dt, idx64=idx64_in)
    plan = sp.spgemm_plan(dA, dB, prec, opts)
    info0 = sp.spgemm_plan_get_info(plan)
    sp.spgemm_symbolic(plan)
    C = sp.alloc_output(plan, idx64_out)
    sp.spgemm_numeric(plan, C)
    if check:
        sp.spgemm_plan_check(plan)
    info = sp.spgemm_plan_get_info(plan)
    torch.cuda.synchronize()
    sp.spgemm_plan_destroy(plan)
    H = C.to_host()
    return (H.row_ptr.numpy().astype(np.int64), H.col.numpy(), H.val.numpy().astype(np.float64),
            info0, info, C)


def assert_parity(A, B, rp, col, val, rows=None, tol=TOL_F64):
    """Compare GPU rows (all, or the listed rows) with the oracle."""
    ref = oracle.spgemm(A, B, rows=rows)
    if rows is None:
        assert np.array_equal(rp, ref.row_ptr), "row_ptr differs"
        assert np.array_equal(col, ref.col), "col differs"
        err = np.abs(val - ref.val)
        bad = err > tol * ref.mag
        assert not bad.any(), f"{bad.sum()} values out of tolerance; worst {(err / np.maximum(ref.mag, 1e-300)).max()}"
        return ref
    for t, i in enumerate(rows):
        g = slice(rp[i], rp[i + 1])
        r = slice(ref.row_ptr[t], ref.row_ptr[t + 1])
        assert rp[i + 1] - rp[i] == ref.row_ptr[t + 1] - ref.row_ptr[t], f"row {i} length differs"
        assert np.array_equal(col[g], ref.col[r]), f"row {i} columns differ"
        err = np.abs(val[g] - ref.val[r])
        assert np.all(err <= tol * ref.mag[r]), f"row {i} values out of tolerance"
    return ref
