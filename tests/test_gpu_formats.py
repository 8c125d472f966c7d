"""Format front-ends on the device (stable radix sort by the new row): CSR transposition (a
matrix's CSC arrays) and COO -> canonical CSR, against scipy's conversions on the host; the CSC
product identity C = A*B in CSC = (B^T A^T) in CSR, against the oracle."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_parity, gpu_or_skip

pytestmark = pytest.mark.gpu
scipy_sparse = pytest.importorskip("scipy.sparse")


@pytest.fixture(autouse=True)
def _gpu():
    gpu_or_skip()


def _sp(M):
    return scipy_sparse.csr_matrix((M.val, M.col, M.row_ptr), shape=(M.rows, M.cols))


@pytest.mark.parametrize("case", ["small", "wide", "tall", "empty_rows", "rmat", "fp32", "idx64", "one_col", "empty"])
def test_transpose_matches_scipy(case):
    import paper_2004_13907_gb300 as sp
    idx64, dtype = False, None
    if case == "small":
        M = synth.random_small(37, 53, 0.2, 1)
    elif case == "wide":        # three radix passes (columns up to 2^17), many tiles
        M = synth.uniform_random(3000, 120_000, 5e-4, seed=2)
    elif case == "tall":
        M = synth.uniform_random(90_000, 700, 2e-3, seed=3)
    elif case == "empty_rows":
        M = synth.from_dense(np.diag(np.arange(1.0, 41.0))[::3])
    elif case == "rmat":
        M = synth.rmat(14, 16, seed=4)
    elif case == "fp32":
        M = synth.uniform_random(2000, 5000, 3e-3, seed=5).astype(np.float32)
        dtype = torch.float32
    elif case == "idx64":
        M = synth.uniform_random(1000, 900, 0.01, seed=6)
        idx64 = True
    elif case == "one_col":
        M = synth.uniform_random(5000, 1, 0.5, seed=7)
    else:
        M = synth.random_small(5, 0, 0.5, 8)
    dM = sp.DeviceCSR.from_host(M, "cuda", dtype=dtype, idx64=idx64)
    T = sp.csr_transpose(dM, idx64=idx64)
    torch.cuda.synchronize()
    ref = _sp(M).T.tocsr()
    ref.sort_indices()
    assert (T.rows, T.cols) == (M.cols, M.rows)
    assert np.array_equal(T.row_ptr.cpu().numpy().astype(np.int64), ref.indptr.astype(np.int64))
    assert np.array_equal(T.col.cpu().numpy(), ref.indices)
    assert np.array_equal(T.val.cpu().numpy(), ref.data.astype(T.val.cpu().numpy().dtype))
    # transposing twice gives M back, bit for bit
    TT = sp.csr_transpose(T)
    assert np.array_equal(TT.row_ptr.cpu().numpy().astype(np.int64), M.row_ptr)
    assert np.array_equal(TT.col.cpu().numpy(), M.col)
    assert np.array_equal(TT.val.cpu().numpy(), M.val)


@pytest.mark.parametrize("seed", [11, 12])
def test_coo_to_csr_from_shuffled_entries(seed):
    import paper_2004_13907_gb300 as sp
    M = synth.uniform_random(20_000, 70_000, 4e-4, seed=seed)
    rows = np.repeat(np.arange(M.rows), np.diff(M.row_ptr)).astype(np.int32)
    perm = np.random.default_rng(seed).permutation(M.nnz)
    C = sp.coo_to_csr(M.rows, M.cols, torch.from_numpy(rows[perm]).cuda(), torch.from_numpy(M.col[perm]).cuda(),
                      torch.from_numpy(M.val[perm]).cuda())
    assert np.array_equal(C.row_ptr.cpu().numpy().astype(np.int64), M.row_ptr)
    assert np.array_equal(C.col.cpu().numpy(), M.col)
    assert np.array_equal(C.val.cpu().numpy(), M.val)


def test_coo_rejects_repeats_and_out_of_range():
    import paper_2004_13907_gb300 as sp
    r = torch.tensor([0, 2, 1, 2], dtype=torch.int32, device="cuda")
    c = torch.tensor([1, 0, 3, 0], dtype=torch.int32, device="cuda")
    v = torch.tensor([1.0, 2.0, 3.0, 4.0], dtype=torch.float64, device="cuda")
    with pytest.raises(sp.SpgemmError) as ei:
        sp.coo_to_csr(3, 4, r, c, v)                       # (2, 0) twice
    assert ei.value.name == "INVALID_CSR"
    with pytest.raises(sp.SpgemmError) as ei:
        sp.coo_to_csr(3, 4, r[:3], torch.tensor([1, 0, 9], dtype=torch.int32, device="cuda"), v[:3])
    assert ei.value.name == "INVALID_CSR"
    C = sp.coo_to_csr(3, 4, r[:3], c[:3], v[:3])
    assert C.row_ptr.cpu().tolist() == [0, 1, 2, 3] and C.col.cpu().tolist() == [1, 3, 0]


def test_csc_product_identity():
    """A and B given by their CSC arrays (the CSR of their transposes): the product's CSC arrays
    come from one CSR product of the views, B^T * A^T, with no conversion."""
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(1500, 2200, 3e-3, seed=21)
    B = synth.uniform_random(2200, 1700, 4e-3, seed=22)
    dA_csc = sp.csr_transpose(sp.DeviceCSR.from_host(A, "cuda"))
    dB_csc = sp.csr_transpose(sp.DeviceCSR.from_host(B, "cuda"))
    Ct = sp.multiply_csc(dA_csc, dB_csc)
    C = sp.csr_transpose(Ct)   # back to CSR for the comparison
    H = C.to_host()
    assert_parity(A, B, H.row_ptr.numpy().astype(np.int64), H.col.numpy(), H.val.numpy())
