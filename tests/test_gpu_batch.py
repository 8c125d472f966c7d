"""Batched products (stacked block-diagonal product) vs the oracle, job by job.

Every job's result view must equal the oracle's product of that job (structure bit-exact,
FP64 values within 1e-12 * sum|a*b|), and the single-product path, for a mix of job shapes:
the batch size distribution (n log-uniform, density log-uniform), empty jobs, rectangular jobs,
jobs with windowed rows, int32 and int64 row pointers; FP32-compensated batches; the CUDA-graph
replay after the values change.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import check_job_rows, gpu_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    gpu_or_skip()


def _jobs(count, seed=0, n_hi=3000):
    jobs = []
    for i in range(count):
        A, B = synth.batch_job(i, seed=seed, n_hi=n_hi)
        jobs.append((A, B))
    return jobs


def _check_job(A, B, C, f32=False):
    ref = oracle.spgemm(A, B)
    rp = C.row_ptr.cpu().numpy().astype(np.int64)
    assert rp.shape == (A.rows + 1,)
    assert np.array_equal(rp, ref.row_ptr)
    assert np.array_equal(C.col.cpu().numpy(), ref.col)
    v = C.val.cpu().numpy().astype(np.float64)
    if f32:
        assert np.all(np.abs(v - ref.val) <= 2.001 * 2.0 ** -24 * np.abs(ref.val) + 2e-12 * ref.mag)
    else:
        assert np.all(np.abs(v - ref.val) <= 1e-12 * ref.mag)


def test_batch_distribution_matches_oracle_per_job():
    import paper_2004_13907_gb300 as sp
    jobs = _jobs(48, seed=0)
    # special jobs: empty, rectangular, windowed rows, int64 row pointers
    jobs.append((synth.random_small(0, 5, 0.5, seed=1), synth.random_small(5, 7, 0.5, seed=2)))
    jobs.append((synth.uniform_random(300, 900, 0.01, seed=3), synth.uniform_random(900, 200, 0.02, seed=4)))
    jobs.append((synth.uniform_random(200, 400, 0.2, seed=5), synth.uniform_random(400, 30_000, 0.05, seed=6)))
    jobs.append((synth.rmat(11, 16, seed=7),) * 2)
    dA = [sp.DeviceCSR.from_host(A, "cuda", idx64=(j % 3 == 1)) for j, (A, _) in enumerate(jobs)]
    dB = [sp.DeviceCSR.from_host(B, "cuda", idx64=(j % 2 == 1)) for j, (_, B) in enumerate(jobs)]
    batch = sp.spgemm_batch(dA, dB)
    batch.check()
    torch.cuda.synchronize()
    info = batch.info()
    assert info["products"] == sum(int(oracle.products_per_row(A, B).sum()) for A, B in jobs)
    for j, (A, B) in enumerate(jobs):
        _check_job(A, B, batch.result(j))
    # the same as the single-product path, job by job
    for j in (0, len(jobs) - 2, len(jobs) - 1):
        single = sp.multiply(dA[j], dB[j])
        got = batch.result(j)
        assert torch.equal(single.col, got.col)
    batch.destroy()


def test_batch_f32c():
    import paper_2004_13907_gb300 as sp
    jobs = [(A.astype(np.float32), B.astype(np.float32)) for A, B in _jobs(24, seed=1)]
    jobs.append((synth.rmat(10, 16, seed=8, dtype=np.float32),) * 2)
    dA = [sp.DeviceCSR.from_host(A, "cuda", dtype=torch.float32) for A, _ in jobs]
    dB = [sp.DeviceCSR.from_host(B, "cuda", dtype=torch.float32) for _, B in jobs]
    batch = sp.spgemm_batch(dA, dB, "f32c")
    batch.check()
    torch.cuda.synchronize()
    for j, (A, B) in enumerate(jobs):
        _check_job(A, B, batch.result(j), f32=True)


def test_batch_graph_replay_after_value_change():
    import paper_2004_13907_gb300 as sp
    jobs = _jobs(16, seed=2)
    dA = [sp.DeviceCSR.from_host(A, "cuda") for A, _ in jobs]
    dB = [sp.DeviceCSR.from_host(B, "cuda") for _, B in jobs]
    batch = sp.spgemm_batch(dA, dB)
    for scale in (2.0, -0.5):
        for t in dA:
            t.val.mul_(scale)
        batch.replay()
        batch.check()
        torch.cuda.synchronize()
    for j, (A, B) in enumerate(jobs):
        A2 = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, A.val * -1.0)
        _check_job(A2, B, batch.result(j))


def test_batch_rejects_bad_job():
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(50, 40, 0.1, seed=9)
    bad = synth.CSR(A.rows, A.cols, A.row_ptr, A.col.copy(), A.val)
    bad.col[0] = 45      # beyond this job's 40 columns (inside the stacked space)
    good = synth.uniform_random(40, 30, 0.1, seed=10)
    dA = [sp.DeviceCSR.from_host(A, "cuda"), sp.DeviceCSR.from_host(bad, "cuda")]
    dB = [sp.DeviceCSR.from_host(good, "cuda")] * 2
    with pytest.raises(sp.SpgemmError) as ei:
        sp.spgemm_batch(dA, dB)
    assert ei.value.name == "INVALID_CSR"


@pytest.mark.parametrize("force_window", [0, 1])
def test_batch_mixed_widths(force_window):
    """Jobs of very different widths in one batch: each row keeps its own job's column count
    (class choice, windowed block counts), including a job wider than one symbolic window
    (2^20 columns) next to narrow jobs with dense rows."""
    import paper_2004_13907_gb300 as sp
    jobs = [
        (synth.uniform_random(300, 60, 0.5, seed=11), synth.uniform_random(60, 900, 0.3, seed=12)),
        (synth.uniform_random(2000, 2000, 0.01, seed=13), synth.uniform_random(2000, 2_500_000, 2e-5, seed=14)),
        (synth.uniform_random(200, 100, 0.6, seed=15), synth.uniform_random(100, 5000, 0.2, seed=16)),
        (synth.laplacian3d(10),) * 2,
    ]
    dA = [sp.DeviceCSR.from_host(A, "cuda") for A, _ in jobs]
    dB = [sp.DeviceCSR.from_host(B, "cuda") for _, B in jobs]
    batch = sp.spgemm_batch(dA, dB, opts=sp.spgemm_opts_default(force_window=force_window))
    batch.check()
    torch.cuda.synchronize()
    for j, (A, B) in enumerate(jobs):
        _check_job(A, B, batch.result(j))
    # every row takes the class it takes alone (the narrow jobs' rows have P far above their
    # own column counts but below the widest job's)
    want = np.zeros(16, dtype=np.int64)
    for a, b in zip(dA, dB):
        plan = sp.spgemm_plan(a, b, opts=sp.spgemm_opts_default(force_window=force_window, general_path=1))
        want += np.array(sp.spgemm_plan_get_info(plan)["sym_class_rows"])
        sp.spgemm_plan_destroy(plan)
    assert np.array_equal(np.array(batch.info()["sym_class_rows"]), want)
    batch.destroy()


def test_autotuned_batch_matches_oracle():
    """The autotuner times every candidate on the batch and returns the fastest options; the batch
    run with them is exact job by job."""
    import paper_2004_13907_gb300 as sp
    jobs = _jobs(40, seed=3)
    jobs.append((synth.rmat(11, 16, seed=12),) * 2)
    jobs.append((synth.laplacian2d(60),) * 2)
    dA = [sp.DeviceCSR.from_host(A, "cuda") for A, _ in jobs]
    dB = [sp.DeviceCSR.from_host(B, "cuda") for _, B in jobs]
    best, rep = sp.spgemm_autotune_batch(dA, dB, reps=1)
    assert len(rep["trials"]) == 9 and rep["best_ms"] <= rep["default_ms"]
    assert min(t["ms"] for t in rep["trials"]) == rep["best_ms"]
    assert best.window_hash_fill in (1024, 2048, 4096) and best.tiny_max in (0, 16, 32)
    batch = sp.spgemm_batch(dA, dB, opts=best)
    batch.check()
    torch.cuda.synchronize()
    for j, (A, B) in enumerate(jobs):
        _check_job(A, B, batch.result(j))
    batch.destroy()


def test_batch_deterministic_mode_equals_exactly_rounded_oracle():
    """fp64_accumulate=2 in a batch: every job's values equal the oracle's correctly rounded sums
    bit for bit (the stacked product routes every row through the exact windowed path)."""
    import paper_2004_13907_gb300 as sp
    jobs = _jobs(24, seed=4)
    jobs.append((synth.rmat(10, 16, seed=9),) * 2)
    dA = [sp.DeviceCSR.from_host(A, "cuda") for A, _ in jobs]
    dB = [sp.DeviceCSR.from_host(B, "cuda") for _, B in jobs]
    batch = sp.spgemm_batch(dA, dB, opts=sp.spgemm_opts_default(fp64_accumulate=2))
    batch.check()
    torch.cuda.synchronize()
    for j, (A, B) in enumerate(jobs):
        ref = oracle.spgemm(A, B, exact_sum=True)
        C = batch.result(j)
        assert np.array_equal(C.row_ptr.cpu().numpy().astype(np.int64), ref.row_ptr)
        assert np.array_equal(C.col.cpu().numpy(), ref.col)
        assert np.array_equal(C.val.cpu().numpy(), ref.val), f"job {j}"
    batch.destroy()


def test_small_job_batch_takes_the_small_path():
    """A batch whose widest job has at most 32,768 columns runs as two kernels over every job's rows
    (each row's bitmap in its own job's column space): every job matches the oracle, and equals
    the same batch through the general row classes column for column."""
    import paper_2004_13907_gb300 as sp
    jobs = _jobs(64, seed=5, n_hi=1000)   # rows of C below 1,024 entries
    jobs.append((synth.random_small(0, 5, 0.5, seed=1), synth.random_small(5, 7, 0.5, seed=2)))
    jobs.append((synth.uniform_random(50, 40, 0.3, seed=9), synth.uniform_random(40, 32_768, 0.001, seed=10)))
    dA = [sp.DeviceCSR.from_host(A, "cuda") for A, _ in jobs]
    dB = [sp.DeviceCSR.from_host(B, "cuda", idx64=(j % 2 == 1)) for j, (_, B) in enumerate(jobs)]
    batch = sp.spgemm_batch(dA, dB)
    batch.check()
    info = batch.info()
    cls = dict(zip(sp._native.NUM_CLASSES, info["num_class_rows"]))
    assert cls["warp1024"] == sum(A.rows for A, _ in jobs)
    ref = sp.spgemm_batch(dA, dB, opts=sp.spgemm_opts_default(general_path=1))
    ref.check()
    torch.cuda.synchronize()
    for j, (A, B) in enumerate(jobs):
        got = batch.result(j)
        _check_job(A, B, got)
        assert torch.equal(got.col, ref.result(j).col)
    batch.destroy()
    ref.destroy()


def test_batch_jobs_from_the_full_distribution():
    """Jobs of the 4,096-job workload as it is drawn (seed 0, n up to 50,000, density up to 1e-2):
    the largest job of all (n = 49,806, about 1.2e10 partial products, 29 GB of C), two jobs near
    8 GB of C and a seeded spread of the rest, stacked in one batch. Jobs with at most 2e7 partial
    products are compared on every row, larger ones on their four heaviest rows and 60 seeded
    others."""
    import paper_2004_13907_gb300 as sp
    rng = np.random.default_rng(31)
    idx = [1313, 2404, 1142] + [int(i) for i in rng.choice(4096, 21, replace=False) if i not in (1313, 2404, 1142)]
    jobs = [synth.batch_job(i, seed=0) for i in idx]
    assert jobs[0][0].rows == 49_806
    dA = [sp.DeviceCSR.from_host(A, "cuda") for A, _ in jobs]
    dB = [sp.DeviceCSR.from_host(B, "cuda") for _, B in jobs]
    batch = sp.spgemm_batch(dA, dB)
    batch.check()
    torch.cuda.synchronize()
    assert batch.info()["products"] == sum(int(oracle.products_per_row(A, B).sum()) for A, B in jobs)
    sampled = sum(check_job_rows(A, B, batch.result(j), rng) for j, (A, B) in enumerate(jobs))
    assert sampled >= 3
    batch.destroy()
    del dA, dB
    torch.cuda.empty_cache()
