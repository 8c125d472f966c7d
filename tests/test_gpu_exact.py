"""Exact fixed-point accumulation of FP64 sums (fp64_accumulate 1: windowed rows; 2: every row,
deterministic) through the C ABI.

* Parity with the oracle: structure bit-exact, values within 1e-12 * sum|a*b| (Alg. 1, Sec. III-A).
* The value of an entry is the correctly rounded sum of its rounded partial products: the same as
  math.fsum (Shewchuk's exactly rounded summation) over the products fl(a_ik * b_kj), computed
  here on the host for sampled rows, and to the oracle's exactly rounded variant for whole
  products in the deterministic mode. So it repeats bit for bit from run to run.
* Rows whose products span more than the fixed-point range, or hold subnormal or non-finite
  values, are redone with FP64 shared atomics; NaN and Inf propagate as in the oracle.
"""

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_parity, gpu_or_skip, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    gpu_or_skip()


def opts(**kw):
    import paper_2004_13907_gb300 as sp
    return sp.spgemm_opts_default(**kw)


def _fsum_rows(A, B, rows):
    """Per listed row: {column: math.fsum of the FP64 products a_ik * b_kj} (host, by definition)."""
    out = {}
    for i in rows:
        acc = {}
        for q in range(A.row_ptr[i], A.row_ptr[i + 1]):
            k, a = int(A.col[q]), float(A.val[q])
            for t in range(B.row_ptr[k], B.row_ptr[k + 1]):
                acc.setdefault(int(B.col[t]), []).append(a * float(B.val[t]))
        out[i] = {j: math.fsum(v) for j, v in acc.items()}
    return out


def _assert_rows_correctly_rounded(A, B, rp, col, val, rows):
    ref = _fsum_rows(A, B, rows)
    for i in rows:
        want = ref[i]
        g = slice(rp[i], rp[i + 1])
        assert list(col[g]) == sorted(want), f"row {i} columns"
        exp = np.array([want[int(j)] for j in col[g]])
        ok = val[g] == exp   # +0 and -0 compare equal
        assert ok.all(), f"row {i}: {(~ok).sum()} entries differ from the correctly rounded sum"


def test_exact_mode_repeats_and_matches_oracle_and_atomic_mode():
    A = synth.rmat(13, 16, seed=11)
    o = opts(force_window=1, fp64_accumulate=1)
    rp, col, val, _, info, _ = run_gpu(A, A, opts=o)
    rp2, col2, val2, *_ = run_gpu(A, A, opts=o)
    assert np.array_equal(val.view(np.uint64), val2.view(np.uint64)), "exact mode is not reproducible"
    assert_parity(A, A, rp, col, val)
    assert info["f32c_rerun_rows"] == 0
    rpa, cola, vala, _, infoa, _ = run_gpu(A, A, opts=opts(force_window=1, fp64_accumulate=0))
    assert np.array_equal(rpa, rp) and np.array_equal(cola, col)
    assert_parity(A, A, rpa, cola, vala)


def test_exact_mode_is_the_correctly_rounded_sum():
    """Signed values with cancellation, every row windowed: each value equals math.fsum of its
    FP64 partial products (sampled rows, including the longest)."""
    A = synth.uniform_random(600, 900, 0.05, seed=12)
    B = synth.uniform_random(900, 700, 0.08, seed=13)
    rp, col, val, _, info, _ = run_gpu(A, B, opts=opts(force_window=1, fp64_accumulate=1))
    assert_parity(A, B, rp, col, val)
    assert info["f32c_rerun_rows"] == 0
    rows = sorted(set(range(0, 600, 37)) | {int(np.argmax(np.diff(A.row_ptr)))})
    _assert_rows_correctly_rounded(A, B, rp, col, val, rows)


def test_long_rows_carry_between_chunks():
    """Rows with far more than 512 A entries (several chunks, limbs normalised between them),
    values of one sign near 1 so the low limbs fill fast, and a signed variant."""
    rng = np.random.default_rng(14)
    n_inner, n = 5000, 6000
    for lo in (0.5, -1.0):
        D = np.zeros((3, n_inner))
        for i, cnt in enumerate((4000, 1500, 600)):
            D[i, rng.choice(n_inner, cnt, replace=False)] = rng.uniform(lo, 1.0, cnt)
        A = synth.from_dense(D)
        B = synth.uniform_random(n_inner, n, 0.02, seed=15, lo=lo, hi=1.0)
        rp, col, val, _, info, _ = run_gpu(A, B, opts=opts(force_window=1, fp64_accumulate=1))
        assert_parity(A, B, rp, col, val)
        assert info["f32c_rerun_rows"] == 0
        _assert_rows_correctly_rounded(A, B, rp, col, val, [0, 1, 2])


def test_integer_values_are_bit_exact():
    """Small integers: every partial sum is exact in FP64, so the oracle's values are exact and the
    exact mode must equal them bit for bit."""
    A = synth.rmat(12, 16, seed=16)
    A = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, np.floor(A.val * 16.0) - 7.0)
    rp, col, val, *_ = run_gpu(A, A, opts=opts(force_window=1, fp64_accumulate=1))
    ref = assert_parity(A, A, rp, col, val)
    assert np.array_equal(val, ref.val)


def test_wide_range_rows_fall_back_to_fp64():
    """Rows mixing 1e-30 and 1 (a range far beyond 2^40) and rows with subnormal products take the
    FP64 shared-atomic path; every value stays within the tolerance."""
    A = synth.rmat(11, 16, seed=17)
    val = A.val.copy()
    lens = np.diff(A.row_ptr)
    heavy = np.argsort(lens)[-6:]
    for t, i in enumerate(heavy):
        s, e = A.row_ptr[i], A.row_ptr[i + 1]
        if t % 2 == 0:
            val[s:(s + e) // 2] *= 1e-30
        else:
            val[s] = 1e-170   # times B values near 1e-160 below: a subnormal product
    A = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, val)
    Bv = synth.rmat(11, 16, seed=17).val.copy()
    Bv[: len(Bv) // 50] *= 1e-160
    B = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, Bv)
    rp, col, val_g, _, info, _ = run_gpu(A, B, opts=opts(force_window=1, fp64_accumulate=1))
    assert_parity(A, B, rp, col, val_g)
    assert info["f32c_rerun_rows"] >= 3


def test_nan_and_inf_propagate():
    A = synth.rmat(10, 16, seed=18)
    val = A.val.copy()
    lens = np.diff(A.row_ptr)
    rows = np.argsort(lens)[-4:]
    val[A.row_ptr[rows[0]]] = np.nan
    val[A.row_ptr[rows[1]]] = np.inf
    A = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, val)
    rp, col, vg, _, info, _ = run_gpu(A, A, opts=opts(force_window=1, fp64_accumulate=1))
    ref = oracle.spgemm(A, A)
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    assert np.array_equal(np.isnan(vg), np.isnan(ref.val))
    assert np.array_equal(np.isposinf(vg), np.isposinf(ref.val))
    fin = np.isfinite(ref.val) & np.isfinite(ref.mag)
    assert np.all(np.abs(vg[fin] - ref.val[fin]) <= 1e-12 * ref.mag[fin])
    assert info["f32c_rerun_rows"] >= 1


@pytest.mark.parametrize("case", ["uniform", "rmat13", "rmat15", "laplacian2d", "rect"])
def test_deterministic_mode_equals_exactly_rounded_oracle(case):
    """fp64_accumulate=2: every value equals the oracle's correctly rounded sum of the entry's
    FP64 products, bit for bit, on every row class's inputs, and repeats on a second run."""
    if case == "uniform":
        A = B = synth.uniform_random(4000, 4000, 2e-3, seed=21)
    elif case == "rmat13":
        A = B = synth.rmat(13, 16, seed=22)
    elif case == "rmat15":
        A = B = synth.rmat(15, 16, seed=3)
    elif case == "laplacian2d":
        A = B = synth.laplacian2d(96)
    else:
        A = synth.uniform_random(1500, 2500, 4e-3, seed=23)
        B = synth.uniform_random(2500, 3100, 3e-3, seed=24)
    o = opts(fp64_accumulate=2)
    rp, col, val, _, info, _ = run_gpu(A, B, opts=o)
    ref = oracle.spgemm(A, B, exact_sum=True)
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    assert info["f32c_rerun_rows"] == 0
    assert np.array_equal(val, ref.val), f"{np.sum(val != ref.val)} values differ from the correctly rounded sums"
    rp2, col2, val2, *_ = run_gpu(A, B, opts=o)
    assert np.array_equal(val.view(np.uint64), val2.view(np.uint64))
