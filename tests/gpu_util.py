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


def compare_all_rows(A, B, C, check, panel_products=2e8):
    """Every row of the device product C = A*B against the oracle, in row panels cut where a
    panel's partial products reach ``panel_products`` (so no panel of C or of the oracle's
    output is large on the host). ``check(ref, rp, col, val, r0, r1)`` asserts one panel: rp are
    C's row offsets of rows [r0, r1) rebased to 0, col/val the panel's entries from the device.
    The oracle computes the next panel while this one is copied and compared."""
    import concurrent.futures as cf
    P = oracle.products_per_row(A, B)
    cs = np.cumsum(P)
    cuts = [0]
    while cuts[-1] < A.rows:
        done = int(cs[cuts[-1] - 1]) if cuts[-1] > 0 else 0
        nxt = int(np.searchsorted(cs, done + panel_products, side="right"))
        cuts.append(min(max(nxt, cuts[-1] + 1), A.rows))
    rp = C.row_ptr.cpu().numpy().astype(np.int64)
    with cf.ThreadPoolExecutor(1) as ex:
        fut = ex.submit(oracle.spgemm, A, B, np.arange(cuts[0], cuts[1], dtype=np.int64))
        for k in range(len(cuts) - 1):
            r0, r1 = cuts[k], cuts[k + 1]
            ref = fut.result()
            if k + 2 < len(cuts):
                fut = ex.submit(oracle.spgemm, A, B, np.arange(r1, cuts[k + 2], dtype=np.int64))
            s, e = int(rp[r0]), int(rp[r1])
            col = C.col[s:e].cpu().numpy()
            val = C.val[s:e].cpu().numpy().astype(np.float64)
            check(ref, rp[r0:r1 + 1] - s, col, val, r0, r1)
    return len(cuts) - 1


def check_job_rows(A, B, C, rng, full_max_products=2e7, sample=60, tol=TOL_F64):
    """A device (or pinned host) product C = A*B against the oracle: every row when the job has
    at most ``full_max_products`` partial products, else its four heaviest rows and ``sample``
    seeded others. Returns True when the rows were sampled."""
    P = oracle.products_per_row(A, B)
    rp = C.row_ptr.cpu().numpy().astype(np.int64)
    if P.sum() <= full_max_products:
        assert_parity(A, B, rp, C.col.cpu().numpy(), C.val.cpu().numpy().astype(np.float64), tol=tol)
        return False
    rows = np.unique(np.concatenate([np.argsort(P)[-4:], rng.choice(A.rows, sample, replace=False)]))
    ref = oracle.spgemm(A, B, rows)
    for t, r in enumerate(rows):
        s, e = int(rp[r]), int(rp[r + 1])
        rs, re = int(ref.row_ptr[t]), int(ref.row_ptr[t + 1])
        assert e - s == re - rs, f"row {r}: {e - s} entries, oracle {re - rs}"
        assert np.array_equal(C.col[s:e].cpu().numpy(), ref.col[rs:re]), f"row {r} columns"
        v = C.val[s:e].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(v - ref.val[rs:re]) <= tol * ref.mag[rs:re]), f"row {r} values"
    return True
