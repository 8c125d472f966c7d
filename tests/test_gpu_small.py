"""The small-product path (F64, at most 65,536 rows and 32,768 columns, default class options: a
warp per row over a bitmap of all columns, one host read) against the oracle: structure bit-exact,
values within 1e-12 * sum|a*b| (Alg. 1, Sec. III-A); rows of C over 1,024 entries fall back to the
general row classes; invalid inputs are reported."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import assert_parity, gpu_or_skip, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    gpu_or_skip()


def opts(**kw):
    import paper_2004_13907_gb300 as sp
    return sp.spgemm_opts_default(**kw)


def _small_taken(info):
    import paper_2004_13907_gb300 as sp
    cls = dict(zip(sp._native.NUM_CLASSES, info["num_class_rows"]))
    return cls["warp1024"] == info["rows"] and sum(info["num_class_rows"]) == info["rows"]


@pytest.mark.parametrize("case", ["uniform10k", "rect", "n1", "n_max", "m_max", "empty_rows", "k0", "lap2d",
                                  "rmat_narrow", "stored_zeros"])
def test_small_path_parity(case):
    if case == "uniform10k":
        A = B = synth.uniform_random(10_000, 10_000, 1e-3, seed=0)
    elif case == "rect":
        A, B = synth.uniform_random(3000, 2500, 4e-3, seed=1), synth.uniform_random(2500, 2000, 6e-3, seed=2)
    elif case == "n1":
        A, B = synth.uniform_random(500, 40, 0.3, seed=3), synth.uniform_random(40, 1, 0.5, seed=4)
    elif case == "n_max":
        A, B = synth.uniform_random(2000, 3000, 2e-3, seed=5), synth.uniform_random(3000, 32_768, 1e-3, seed=6)
    elif case == "m_max":
        A, B = synth.uniform_random(65_536, 4000, 1e-3, seed=7), synth.uniform_random(4000, 5000, 2e-3, seed=8)
    elif case == "empty_rows":
        A = synth.from_dense(np.diag(np.arange(1.0, 301.0))[::7])
        B = synth.uniform_random(300, 900, 0.02, seed=9)
    elif case == "k0":
        A, B = synth.random_small(40, 0, 0.5, 10), synth.random_small(0, 30, 0.5, 11)
    elif case == "lap2d":
        A = B = synth.laplacian2d(128)
    elif case == "rmat_narrow":
        A = B = synth.rmat(11, 8, seed=12)
    else:
        D = np.array([[1.0, 1.0, 0.0], [0.0, 2.0, 5.0]])
        A = synth.from_dense(D, pattern=np.array([[True, True, False], [True, True, True]]))
        B = synth.from_dense(np.array([[1.0, 3.0], [-1.0, 0.0], [0.0, 0.0]]),
                             pattern=np.array([[True, False], [True, True], [False, True]]))
    rp, col, val, _, info, _ = run_gpu(A, B)
    assert_parity(A, B, rp, col, val)
    if A.rows > 0 and B.cols > 0:
        assert _small_taken(info) or case == "rmat_narrow"
    rp2, col2, val2, *_ = run_gpu(A, B, opts=opts(general_path=1))
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)


def test_long_rows_fall_back_to_the_general_path():
    """A row of C with more than 1,024 entries: the plan counts again through the row classes."""
    rng = np.random.default_rng(13)
    D = np.zeros((50, 400))
    D[3, :] = rng.uniform(-1, 1, 400)          # a dense row of A
    D[10:, :8] = rng.uniform(-1, 1, (40, 8))
    A = synth.from_dense(D)
    B = synth.uniform_random(400, 20_000, 0.01, seed=14)   # row 3 of C: about 13,000 entries
    rp, col, val, _, info, _ = run_gpu(A, B)
    assert_parity(A, B, rp, col, val)
    assert not _small_taken(info)
    assert int(np.diff(rp).max()) > 1024


def test_small_path_reports_invalid_inputs():
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(60, 50, 0.1, seed=15)
    B = synth.uniform_random(50, 70, 0.1, seed=16)
    bad = []
    col = A.col.copy()
    r = int(np.argmax(np.diff(A.row_ptr) >= 2))
    s = A.row_ptr[r]
    col[s], col[s + 1] = col[s + 1], col[s]                        # A row not sorted
    bad.append((synth.CSR(A.rows, A.cols, A.row_ptr, col, A.val), B))
    col = A.col.copy()
    col[5] = 50                                                    # A column outside B's rows
    bad.append((synth.CSR(A.rows, A.cols, A.row_ptr, col, A.val), B))
    bcol = B.col.copy()
    bcol[7] = 999                                                  # B column outside n
    bad.append((A, synth.CSR(B.rows, B.cols, B.row_ptr, bcol, B.val)))
    rpa = A.row_ptr.copy()
    rpa[10], rpa[11] = rpa[11], rpa[10]                            # decreasing row pointers
    bad.append((synth.CSR(A.rows, A.cols, rpa, A.col, A.val), B))
    for Ai, Bi in bad:
        dA, dB = sp.DeviceCSR.from_host(Ai, "cuda"), sp.DeviceCSR.from_host(Bi, "cuda")
        with pytest.raises(sp.SpgemmError) as ei:
            plan = sp.spgemm_plan(dA, dB)
            sp.spgemm_symbolic(plan)
        assert ei.value.name == "INVALID_CSR"
    rp, col, val, *_ = run_gpu(A, B)
    assert_parity(A, B, rp, col, val)
