"""The torch generator builds the same matrices as the numpy one (bit for bit, on the CPU here),
so the bench can build the batch-distribution jobs in device memory and still measure the inputs
the tests and the oracle use."""

import numpy as np
import pytest
import torch

import synth
from synth import torch_gen


@pytest.mark.parametrize("m,n,d,seed", [(0, 5, 0.1, 1), (1, 1, 0.5, 2), (50, 400, 0.01, 3), (300, 300, 0.05, 4),
                                        (1000, 7000, 1e-3, 5), (2000, 2000, 3e-4, 6)])
def test_uniform_random_matches_numpy(m, n, d, seed):
    ref = synth.uniform_random(m, n, d, seed, stream_base=40)
    rp, col, val = torch_gen.uniform_random(m, n, d, seed, stream_base=40, device="cpu")
    assert np.array_equal(rp.numpy(), ref.row_ptr)
    assert np.array_equal(col.numpy(), ref.col)
    assert np.array_equal(val.numpy().view(np.uint64), ref.val.view(np.uint64))


@pytest.mark.parametrize("i", [0, 1, 7, 33, 100, 257])
def test_batch_job_matches_numpy(i):
    n, d = synth.batch_job_params(i, 0)
    if n > 8000:
        pytest.skip("large job (kept out of the CPU suite for time)")
    A, B = synth.batch_job(i, 0)
    n2, tA, tB = torch_gen.batch_job(i, 0, device="cpu")
    assert n2 == n
    for ref, (rp, col, val) in ((A, tA), (B, tB)):
        assert np.array_equal(rp.numpy(), ref.row_ptr)
        assert np.array_equal(col.numpy(), ref.col)
        assert np.array_equal(val.numpy(), ref.val)


def test_counter_stream_matches_numpy():
    c = np.array([0, 1, 2, 3, 1 << 40, (1 << 62) + 5], dtype=np.uint64)
    want = synth.counter_u64(9, 123, c).view(np.int64)
    got = torch_gen.counter_u64(9, 123, torch.from_numpy(c.view(np.int64))).numpy()
    assert np.array_equal(got, want)
