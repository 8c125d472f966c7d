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


def test_traffic_lookup_reads_the_profile_only_for_the_current_source(tmp_path):
    """The bench's roofline traffic comes from a committed ncu summary (DRAM bytes per algorithmic
    byte of the windowed pass) whose recorded source hash matches the kernel file as it is; a stale
    summary gives None."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2004_13907_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k_window.cu").write_text("__global__ void k() {}\n")
    sha = hashlib.sha256((csrc / "k_window.cu").read_bytes()).hexdigest()[:16]
    prof = tmp_path / "profiles" / "k_num_window_rmat17.md"
    prof.write_text(f"# k\n\n- kernel source sha256[:16]: `{sha}`\n- dram bytes per algorithmic byte: 0.25\n")
    assert bench._traffic(4000, root=str(tmp_path)) == 1000
    (csrc / "k_window.cu").write_text("__global__ void k() { }\n")
    assert bench._traffic(4000, root=str(tmp_path)) is None


def test_committed_window_profile_parses():
    """The committed small-case summary of the windowed pass carries a source hash and a ratio of
    DRAM bytes to algorithmic bytes."""
    import re
    text = open(os.path.join(ROOT, "profiles", "k_num_window_rmat17.md")).read()
    assert re.search(r"- kernel source sha256\[:16\]: `[0-9a-f]{16}`", text)
    assert re.search(r"- dram bytes per algorithmic byte: [0-9.]+", text)


def test_fp64_pipe_fraction():
    """Two FP64 operations per partial product against 2 lanes per clock per SM."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench._fp64_pipe(20_919_618_292, 241.0, 152, 2070.0)
    assert r["fp64_peak_ops_per_s"] == 2.0 * 152 * 2070e6
    assert abs(r["fp64_ops_per_s"] - 2 * 20_919_618_292 / 0.241) < 1.0
    assert abs(r["fp64_frac"] - 0.2757) < 1e-3
    assert abs(r["fp64_floor_ms"] - 66.49) < 0.01
    assert bench._fp64_pipe(1, 1.0, 1, None)["fp64_peak_ops_per_s"] == 2.0 * 2070e6


def test_algorithmic_bytes_follow_the_value_width():
    """The numeric pass's algorithmic bytes: A rows (8 per row pointer pair), per A entry its column,
    value and the named B row's bounds, per partial product the gathered B column and value, per
    entry of C its column and value, with 8-byte (FP64) or 4-byte (FP32) values."""
    sys.path.insert(0, ROOT)
    import bench
    info = {"num_class_rows": [2, 3, 0, 0] + [7] * 12, "num_class_annz": [10, 20, 0, 0] + [5] * 12,
            "num_class_products": [100, 300, 0, 0] + [9] * 12, "num_class_cnnz": [40, 60, 0, 0] + [3] * 12,
            "products": 400 + 9 * 12, "nnz_c": 100 + 3 * 12}
    # windowed classes only (the first four)
    b64, p64 = bench._window_bytes(info, 8)
    b32, p32 = bench._window_bytes(info, 4)
    assert p64 == p32 == 400
    assert b64 == 8 * 5 + (12 + 8) * 30 + (4 + 8) * 400 + (4 + 8) * 100
    assert b32 == 8 * 5 + (12 + 4) * 30 + (4 + 4) * 400 + (4 + 4) * 100
    assert bench._window_bytes(info) == (b64, p64)
    # a whole pass: every class, both row pointer arrays
    m = 50
    annz = 30 + 5 * 12
    n64 = bench._numeric_bytes(info, m, 8)
    n32 = bench._numeric_bytes(info, m, 4)
    assert n64 == 4 * (m + 1) + 12 * annz + 8 * annz + 12 * info["products"] + 8 * (m + 1) + 12 * info["nnz_c"]
    assert n64 - n32 == 4 * (annz + info["products"] + info["nnz_c"])
    assert bench._vbytes("f32c") == 4 and bench._vbytes("f64") == 8
