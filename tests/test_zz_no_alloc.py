"""spgemm_multiply_noalloc, the entry point for callers that cannot allocate device memory
(services holding a fixed device reservation, real-time loops that must not block in an
allocator): its output must match the regular plan/symbolic/numeric path, called through the
C ABI, on two calls in a row that reuse its fixed scratch array. This file is collected last
on purpose."""

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


def _csr(rows, cols, row_ptr, col, val):
    return synth.CSR(rows, cols, np.asarray(row_ptr, np.int64), np.asarray(col, np.int32),
                     np.asarray(val, np.float64))


def test_noalloc_row_entry_limit_4096_and_4097():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_13907_gb300 as sp
    A = _csr(1, 1, [0, 1], [0], [2.0])
    for n, ok in ((4096, True), (4097, False)):
        B = _csr(1, n, [0, n], np.arange(n), np.linspace(-1.0, 1.0, n))
        dA, dB = sp.DeviceCSR.from_host(A, "cuda"), sp.DeviceCSR.from_host(B, "cuda")
        if ok:
            got = _noalloc(sp, dA, dB, n)
            assert int(got.col.numel()) == n
            assert np.array_equal(got.col.cpu().numpy(), np.arange(n))
            assert np.array_equal(got.val.cpu().numpy(), 2.0 * B.val)   # one exact product per entry
        else:
            with pytest.raises(sp.SpgemmError) as ei:
                _noalloc(sp, dA, dB, n)
            assert ei.value.name == "UNSUPPORTED"


def test_noalloc_rejects_out_of_range_columns():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_13907_gb300 as sp
    B = _csr(2, 3, [0, 2, 3], [0, 2, 1], [1.0, 2.0, 3.0])
    bad_a = _csr(1, 2, [0, 1], [5], [1.0])            # column of A >= B.rows
    good_a = _csr(1, 2, [0, 2], [0, 1], [1.0, 1.0])
    bad_b = _csr(2, 3, [0, 2, 3], [0, 7, 1], [1.0, 2.0, 3.0])   # column of B >= B.cols
    for A_, B_ in ((bad_a, B), (good_a, bad_b)):
        dA, dB = sp.DeviceCSR.from_host(A_, "cuda"), sp.DeviceCSR.from_host(B_, "cuda")
        with pytest.raises(sp.SpgemmError) as ei:
            _noalloc(sp, dA, dB, 16)
        assert ei.value.name == "INVALID_CSR"
    # the scratch array is usable again after a refused call
    dA, dB = sp.DeviceCSR.from_host(good_a, "cuda"), sp.DeviceCSR.from_host(B, "cuda")
    got = _noalloc(sp, dA, dB, 16)
    assert np.array_equal(got.col.cpu().numpy(), [0, 1, 2])
    assert np.array_equal(got.val.cpu().numpy(), [1.0, 3.0, 2.0])
