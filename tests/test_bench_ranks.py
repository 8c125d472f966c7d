"""The multi-rank path of bench.py on the CPU: two gloo ranks (world size 2, 127.0.0.1) agree on
the slowest rank's step time, the whole-job value counts every rank's replica, and the reference
arm does no work on ranks other than 0. No GPU and no CUDA call."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    step_ms = [10.0, 25.0][rank]                 # rank 1 is the slow replica
    ms = bench._max_over_ranks(step_ms, dist, "cpu")
    value = bench._job_gflops(1_000_000, world, ms)
    ws, r, _ = bench._dist()
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, value, ws, r))


def test_two_gloo_ranks_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, ws, r in res:
        assert ms == 25.0 and ws == 2 and r == rank
        assert value == pytest.approx(2.0 * 1_000_000 * 2 / 25e-3 / 1e9)


def test_reference_arm_is_rank0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    line, rank = bench.run_reference(None)       # returns before touching the workload
    assert line is None and rank == 1
