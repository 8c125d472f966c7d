"""spgemm_multiply_noalloc, the entry point for callers that cannot allocate device memory
(graph capture, fixed device reservations, real-time loops): its output must match the
regular plan/symbolic/numeric path, called through the C ABI, on two calls in a row that
reuse its fixed scratch array. This file is collected last on purpose."""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _check_same(A, B, got, want):
    assert np.array_equal(got.row_ptr.cpu().numpy().astype(np.int64), want.row_ptr.cpu().numpy().astype(np.int64))
    assert np.array_equal(got.col.cpu().numpy(), want.col.cpu().numpy())
    ref = oracle.spgemm(A, B)
    diff = np.abs(got.val.cpu().numpy() - want.val.cpu().numpy())
    assert np.all(diff <= 2e-12 * ref.mag)   # each side within 1e-12 * sum|a*b| of the exact sum


def _noalloc(sp, dA, dB, cap, idx64=False):
    C = sp.DeviceCSR(dA.rows, dB.cols,
                     torch.empty(dA.rows + 1, dtype=torch.int64 if idx64 else torch.int32, device="cuda"),
                     torch.empty(cap, dtype=torch.int32, device="cuda"),
                     torch.empty(cap, dtype=torch.float64, device="cuda"))
    nnz = sp.spgemm_multiply_noalloc(dA, dB, C)
    torch.cuda.synchronize()
    return sp.DeviceCSR(C.rows, C.cols, C.row_ptr, C.col[:nnz], C.val[:nnz])


def test_noalloc_matches_regular_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_13907_gb300 as sp
    cases = [
        (synth.uniform_random(3000, 2500, 3e-3, seed=31), synth.uniform_random(2500, 4000, 4e-3, seed=32)),
        (synth.rmat(12, 16, seed=33), None),
    ]
    for A, B in cases:
        B = A if B is None else B
        dA = sp.DeviceCSR.from_host(A, "cuda")
        dB = sp.DeviceCSR.from_host(B, "cuda", idx64=True)
        want = sp.multiply(dA, dB, check=True)
        torch.cuda.synchronize()
        for _ in range(2):   # the second call reuses the same scratch array
            got = _noalloc(sp, dA, dB, want.nnz + 17)
            _check_same(A, B, got, want)


def test_noalloc_capacity_and_limits():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(500, 500, 1e-2, seed=34)
    dA = sp.DeviceCSR.from_host(A, "cuda")
    want = sp.multiply(dA, dA)
    with pytest.raises(sp.SpgemmError) as ei:
        _noalloc(sp, dA, dA, 10)
    assert ei.value.name == "INVALID_ARG" and ei.value.nnz_c == want.nnz
    got = _noalloc(sp, dA, dA, want.nnz, idx64=True)
    _check_same(A, A, got, want)
    big = synth.uniform_random(1 << 16 | 1, 10, 0.1, seed=35)
    dbig = sp.DeviceCSR.from_host(big, "cuda")
    dB = sp.DeviceCSR.from_host(synth.uniform_random(10, 10, 0.5, seed=36), "cuda")
    with pytest.raises(sp.SpgemmError) as ei:
        _noalloc(sp, dbig, dB, 10)
    assert ei.value.name == "UNSUPPORTED"
