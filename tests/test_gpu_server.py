"""The serving layer: jobs submitted one at a time, run in fused batches.

Each job's result from the server, where it ran inside a batch with other jobs, must be the
same as the job run alone: structure bit-exact, FP64 values within 1e-12 * sum|a*b| of the
oracle on both sides. Also: admission against the memory cap (a batch too big for the cap is
split, a job too big alone is rejected, memory returns to zero once results are released), a
paused server's bounded wait returning TIMEOUT, the completion queue, an invalid job failing alone, submissions from
several host threads, FP32-compensated serving, and the statistics.
"""

import threading

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


def _mix(count, seed):
    jobs = [synth.batch_job(i, seed=seed, n_hi=2500) for i in range(count)]
    jobs.append((synth.laplacian3d(12),) * 2)
    jobs.append((synth.laplacian2d(40),) * 2)
    jobs.append((synth.random_small(0, 6, 0.5, seed=seed + 1), synth.random_small(6, 9, 0.5, seed=seed + 2)))
    jobs.append((synth.uniform_random(150, 300, 0.2, seed=seed + 3), synth.uniform_random(300, 20_000, 0.05, seed=seed + 4)))
    jobs.append((synth.rmat(10, 16, seed=seed + 5),) * 2)
    return jobs


def _to_dev(sp, jobs, dtype=torch.float64):
    return [(sp.DeviceCSR.from_host(A, "cuda", dtype=dtype, idx64=(j % 3 == 2)),
             sp.DeviceCSR.from_host(B, "cuda", dtype=dtype, idx64=(j % 2 == 1))) for j, (A, B) in enumerate(jobs)]


def _same_as_alone(A, B, got, alone, f32=False):
    ref = oracle.spgemm(A, B)
    rp = got.row_ptr.cpu().numpy().astype(np.int64)
    assert np.array_equal(rp, alone.row_ptr.cpu().numpy().astype(np.int64))
    assert np.array_equal(rp, ref.row_ptr)
    assert np.array_equal(got.col.cpu().numpy(), alone.col.cpu().numpy())
    assert np.array_equal(got.col.cpu().numpy(), ref.col)
    v = got.val.cpu().numpy().astype(np.float64)
    w = alone.val.cpu().numpy().astype(np.float64)
    if f32:
        lim = 2.001 * 2.0 ** -24 * np.abs(ref.val) + 2e-12 * ref.mag
        assert np.all(np.abs(v - ref.val) <= lim) and np.all(np.abs(w - ref.val) <= lim)
    else:
        assert np.all(np.abs(v - ref.val) <= 1e-12 * ref.mag)
        assert np.all(np.abs(v - w) <= 2e-12 * ref.mag)


def test_results_alone_equal_results_in_the_mix():
    import paper_2004_13907_gb300 as sp
    jobs = _mix(40, seed=50)
    dev = _to_dev(sp, jobs)
    alone = [sp.multiply(dA, dB) for dA, dB in dev]
    torch.cuda.synchronize()
    with sp.Server(batch_window_us=20_000, start_paused=1) as srv:
        ids = [srv.submit(dA, dB) for dA, dB in dev]
        srv.resume()
        infos = [srv.wait(i, timeout=120) for i in ids]
        assert max(inf["batch_jobs"] for inf in infos) > 1, "no job ran in a fused batch"
        for (A, B), i, inf, ref in zip(jobs, ids, infos, alone):
            assert inf["state"] == "done" and inf["nnz"] == ref.col.numel()
            _same_as_alone(A, B, srv.result(i), ref)
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 0 and st["rejected"] == 0
        assert st["products"] == sum(int(oracle.products_per_row(A, B).sum()) for A, B in jobs)
        assert 0 < st["latency_p50_ms"] <= st["latency_p99_ms"] <= st["latency_max_ms"]
        assert st["mean_batch_jobs"] > 1
        for i in ids:
            srv.release(i)
        assert srv.stats()["bytes_in_use"] == 0


def test_paused_server_wait_times_out_then_runs():
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(700, 600, 0.01, seed=60)
    B = synth.uniform_random(600, 800, 0.01, seed=61)
    dA, dB = sp.DeviceCSR.from_host(A, "cuda"), sp.DeviceCSR.from_host(B, "cuda")
    with sp.Server(start_paused=1) as srv:
        j = srv.submit(dA, dB)
        with pytest.raises(sp.SpgemmError) as ei:
            srv.wait(j, timeout=0.3)
        assert ei.value.name == "TIMEOUT"
        assert srv.poll(j)["state"] == "queued"
        with pytest.raises(sp.SpgemmError) as ei:
            srv.result(j)
        assert ei.value.name == "NOT_READY"
        with pytest.raises(sp.SpgemmError) as ei:
            srv.release(j)
        assert ei.value.name == "NOT_READY"
        srv.resume()
        inf = srv.wait(j, timeout=60)
        assert inf["state"] == "done" and inf["latency_ms"] >= 300
        _same_as_alone(A, B, srv.result(j), sp.multiply(dA, dB))
        srv.release(j)
        with pytest.raises(sp.SpgemmError):
            srv.poll(j)


def test_completion_queue_returns_every_job_once_in_finish_order():
    """wait_any hands out each finished job exactly once (a rejected one too), times out while
    nothing has finished, and skips a job released before it came out."""
    import paper_2004_13907_gb300 as sp
    jobs = [synth.batch_job(i, seed=71, n_hi=2000) for i in range(24)]
    dev = _to_dev(sp, jobs)
    big = synth.uniform_random(3000, 3000, 0.05, seed=72)
    dbig = sp.DeviceCSR.from_host(big, "cuda")
    with sp.Server(start_paused=1, mem_cap_bytes=8 << 20, host_panels=0) as srv:
        ids = [srv.submit(dA, dB) for dA, dB in dev]
        rej = srv.submit(dbig, dbig)          # inputs over the 8 MB cap on their own: rejected
        assert srv.wait_any(timeout=0.2) is None
        srv.resume()
        first = srv.wait(ids[0], timeout=60)
        assert first["state"] == "done"
        srv.release(ids[0])                    # released before wait_any returned it: skipped
        seen = []
        while len(seen) < len(ids):
            j = srv.wait_any(timeout=60)
            assert j is not None
            seen.append(j)
            if j != rej:
                A, B = jobs[ids.index(j)]
                dA, dB = dev[ids.index(j)]
                _same_as_alone(A, B, srv.result(j), sp.multiply(dA, dB))
            srv.release(j)
        assert sorted(seen) == sorted(ids[1:] + [rej])
        assert srv.wait_any(timeout=0.05) is None
        assert srv.wait_any(timeout=0) is None


def test_admission_splits_batches_and_rejects_oversized_jobs():
    import paper_2004_13907_gb300 as sp
    jobs = [synth.batch_job(i, seed=70, n_lo=800, n_hi=1200, d_lo=0.008, d_hi=0.012) for i in range(6)]
    dev = _to_dev(sp, jobs)
    with sp.Server() as srv:   # the exact bytes each job needs alone
        needs = []
        for dA, dB in dev:
            j = srv.submit(dA, dB)
            needs.append(srv.wait(j, timeout=60)["needed_bytes"])
            srv.release(j)
    cap = int(1.5 * max(needs))
    # small inputs, large output: its preparation fits the cap, its exact size does not
    dbig = sp.DeviceCSR.from_host(synth.uniform_random(1500, 16, 0.9, seed=71), "cuda")
    dbigB = sp.DeviceCSR.from_host(synth.uniform_random(16, 1500, 0.9, seed=72), "cuda")
    # inputs alone over the cap: rejected from its sizes, before any device work
    dhuge = sp.DeviceCSR.from_host(synth.uniform_random(20_000, 20_000, 1e-3, seed=73), "cuda")
    with sp.Server(mem_cap_bytes=cap, start_paused=1, batch_window_us=50_000, host_panels=0) as srv:
        ids = [srv.submit(dA, dB) for dA, dB in dev]
        jbig = srv.submit(dbig, dbigB)
        jhuge = srv.submit(dhuge, dhuge)
        srv.resume()
        for (A, B), (dA, dB), i in zip(jobs, dev, ids):
            inf = srv.wait(i, timeout=120)
            assert inf["state"] == "done" and inf["needed_bytes"] <= cap
            _same_as_alone(A, B, srv.result(i), sp.multiply(dA, dB))
            srv.release(i)      # frees room for the next batch under the cap
        with pytest.raises(sp.SpgemmError) as ei:
            srv.wait(jbig, timeout=120)
        assert ei.value.name == "REJECTED"
        for j in (jbig, jhuge):
            inf = srv.poll(j)
            assert inf["state"] == "rejected" and inf["needed_bytes"] > cap
        st = srv.stats()
        assert st["splits"] >= 1 and st["rejected"] == 2 and st["completed"] == len(jobs)
        assert st["bytes_peak"] <= cap
        srv.release(jbig)
        srv.release(jhuge)
        assert srv.stats()["bytes_in_use"] == 0


def test_invalid_job_fails_alone():
    import paper_2004_13907_gb300 as sp
    jobs = _mix(6, seed=80)
    dev = _to_dev(sp, jobs)
    bad = synth.uniform_random(50, 40, 0.2, seed=81)
    bad.col = bad.col.copy()
    r = int(np.argmax(np.diff(bad.row_ptr) > 0))
    bad.col[bad.row_ptr[r + 1] - 1] = 45      # the last entry of a non-empty row, past A.cols
    dbad = sp.DeviceCSR.from_host(bad, "cuda")
    dB = sp.DeviceCSR.from_host(synth.uniform_random(40, 30, 0.2, seed=82), "cuda")
    with sp.Server(start_paused=1, batch_window_us=50_000) as srv:
        ids = [srv.submit(dA, dBj) for dA, dBj in dev[:3]]
        jb = srv.submit(dbad, dB)
        ids += [srv.submit(dA, dBj) for dA, dBj in dev[3:]]
        srv.resume()
        with pytest.raises(sp.SpgemmError) as ei:
            srv.wait(jb, timeout=120)
        assert ei.value.name == "INVALID_CSR"
        for (A, B), (dA, dBj), i in zip(jobs, dev, ids):
            assert srv.wait(i, timeout=120)["state"] == "done"
            _same_as_alone(A, B, srv.result(i), sp.multiply(dA, dBj))
        assert srv.stats()["failed"] == 1


def test_submit_from_several_threads():
    import paper_2004_13907_gb300 as sp
    jobs = _mix(30, seed=90)
    dev = _to_dev(sp, jobs)
    alone = [sp.multiply(dA, dB) for dA, dB in dev]
    torch.cuda.synchronize()
    errors = []
    with sp.Server(batch_window_us=500, num_streams=3) as srv:
        def worker(k):
            try:
                mine = list(range(k, len(jobs), 4))
                ids = [srv.submit(*dev[t]) for t in mine]
                for t, i in zip(mine, ids):
                    srv.wait(i, timeout=120)
                    got = srv.result(i)
                    assert torch.equal(got.col, alone[t].col)
                    assert torch.equal(got.row_ptr.to(torch.int64), alone[t].row_ptr.to(torch.int64))
                    srv.release(i)
            except Exception as e:   # reported by the main thread
                errors.append(e)
        threads = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors[0]
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["bytes_in_use"] == 0


def test_f32c_server():
    import paper_2004_13907_gb300 as sp
    jobs = [(A.astype(np.float32), B.astype(np.float32)) for A, B in _mix(12, seed=100)]
    dev = _to_dev(sp, jobs, dtype=torch.float32)
    with sp.Server(prec="f32c", start_paused=1, batch_window_us=20_000) as srv:
        ids = [srv.submit(dA, dB) for dA, dB in dev]
        srv.resume()
        for (A, B), (dA, dB), i in zip(jobs, dev, ids):
            assert srv.wait(i, timeout=120)["state"] == "done"
            _same_as_alone(A, B, srv.result(i), sp.multiply(dA, dB, prec="f32c"), f32=True)


def test_small_jobs_overtake_a_large_one_for_a_bounded_time():
    """With a paused queue holding a large job followed by small ones, the small jobs run first
    (they overtake it), and with max_defer_ms=0 strict arrival order holds."""
    import paper_2004_13907_gb300 as sp
    big = synth.uniform_random(10_000, 10_000, 2e-2, seed=110)     # about 4e8 expected products
    smalls = [synth.batch_job(i, seed=111, n_lo=200, n_hi=400) for i in range(5)]
    dbig = sp.DeviceCSR.from_host(big, "cuda")
    dsm = [(sp.DeviceCSR.from_host(A, "cuda"), sp.DeviceCSR.from_host(B, "cuda")) for A, B in smalls]
    for defer, small_first in ((10_000, True), (0, False)):
        with sp.Server(start_paused=1, num_streams=1, batch_window_us=0, max_batch_jobs=1,
                       max_defer_ms=defer) as srv:
            jb = srv.submit(dbig, dbig)
            js = [srv.submit(a, b) for a, b in dsm]
            srv.resume()
            ib = srv.wait(jb, timeout=120)
            iss = [srv.wait(j, timeout=120) for j in js]
            if small_first:
                assert all(x["batch"] < ib["batch"] for x in iss)
            else:
                assert all(x["batch"] > ib["batch"] for x in iss)
            for (A, B), (a, b), j in zip(smalls, dsm, js):
                _same_as_alone(A, B, srv.result(j), sp.multiply(a, b))


def test_job_over_the_cap_runs_as_row_panels():
    """A job whose exact size exceeds the cap runs as row panels, each under a quarter of the cap,
    into a pinned host result equal to the oracle's product; device memory never exceeds the cap."""
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(1500, 16, 0.9, seed=120)
    B = synth.uniform_random(16, 1500, 0.9, seed=121)
    dA, dB = sp.DeviceCSR.from_host(A, "cuda"), sp.DeviceCSR.from_host(B, "cuda")
    cap = 6 << 20          # the product's output alone is about 27 MB
    small = synth.batch_job(0, seed=122, n_lo=300, n_hi=400)
    ds = (sp.DeviceCSR.from_host(small[0], "cuda"), sp.DeviceCSR.from_host(small[1], "cuda"))
    with sp.Server(mem_cap_bytes=cap) as srv:
        j = srv.submit(dA, dB)
        js = srv.submit(*ds)
        inf = srv.wait(j, timeout=300)
        assert inf["state"] == "done" and inf["result_on_host"] == 1 and inf["panels"] > 4
        C = srv.result(j)
        assert C.col.device.type == "cpu"
        ref = oracle.spgemm(A, B)
        assert np.array_equal(C.row_ptr.numpy(), ref.row_ptr)
        assert np.array_equal(C.col.numpy(), ref.col)
        assert np.all(np.abs(C.val.numpy() - ref.val) <= 1e-12 * ref.mag)
        srv.wait(js, timeout=60)
        _same_as_alone(*small, srv.result(js), sp.multiply(*ds))
        st = srv.stats()
        assert st["bytes_peak"] <= cap and st["completed"] == 2
        srv.release(j)
        srv.release(js)
        assert srv.stats()["bytes_in_use"] == 0


def test_serving_the_largest_jobs_of_the_request_stream():
    """Requests as the 20,000-request workload draws them, under its 32 GB cap: the four largest
    jobs of the 512 it cycles through (up to n = 47,624 and 24 GB of C), the largest 3D Laplacian
    (g = 128) and 24 other jobs of the 512, served together. Each result is checked and released
    as it comes out of the completion queue (the cap holds one large result at a time): every row
    of a job with at most 2e7 partial products, the four heaviest rows and 60 seeded others of a
    larger one."""
    import paper_2004_13907_gb300 as sp
    rng = np.random.default_rng(91)
    big = [226, 52, 56, 154]
    others = [int(i) for i in rng.choice(512, 30, replace=False) if int(i) not in big][:24]
    jobs = [synth.batch_job(i, seed=0) for i in big + others]
    jobs.append((synth.laplacian3d(128),) * 2)
    assert jobs[0][0].rows == 47_624
    dev = [(sp.DeviceCSR.from_host(A, "cuda"), sp.DeviceCSR.from_host(B, "cuda")) for A, B in jobs]
    cap = 32 << 30
    with sp.Server(mem_cap_bytes=cap, start_paused=1) as srv:
        ids = [srv.submit(dA, dB) for dA, dB in dev]
        srv.resume()
        sampled = 0
        for _ in ids:
            j = srv.wait_any(timeout=300)
            assert j is not None, "no job finished for 300 s"
            assert srv.poll(j)["state"] == "done"
            A, B = jobs[ids.index(j)]
            sampled += check_job_rows(A, B, srv.result(j), rng)
            srv.release(j)
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 0 and st["rejected"] == 0
        assert st["bytes_peak"] <= cap and st["bytes_in_use"] == 0
    assert sampled >= 4
