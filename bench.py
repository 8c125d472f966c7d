#!/usr/bin/env python3
"""SpGEMM throughput on GB300: C = A*A on synthetic matrices shaped like the paper's
workloads (the paper evaluates C = A^2, Sec. V).

One step = the whole product for every matrix of the workload: plan (validation, product
count, row classes), symbolic pass, allocation of C, numeric pass. The metric is GFLOP/s
= 2 * (number of partial products) / time. Default workload: the 2D 5-point Laplacian on a
1024 x 1024 grid and the R-MAT graph with 2^20 vertices and average degree 16, both FP64.

Prints ONE JSON line (rank 0). ``--impl reference`` times the CPU oracle instead (rank 0
only), on a bounded row sample of the same workload each step.
"""

from __future__ import annotations

import argparse
import csv
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "SpGEMM GFLOP/s (2 x intermediate products / s)"
UNIT = "GFLOP/s"

WORKLOADS = {
    # name -> list of (matrix name, generator, precision)
    "lap2d1024+rmat20": [("lap2d_1024", lambda: synth.laplacian2d(1024), "f64"),
                         ("rmat_2e20_deg16", lambda: synth.rmat(20, 16, seed=0), "f64")],
    "lap2d1024": [("lap2d_1024", lambda: synth.laplacian2d(1024), "f64")],
    "rmat20": [("rmat_2e20_deg16", lambda: synth.rmat(20, 16, seed=0), "f64")],
    "rmat20_f32c": [("rmat_2e20_deg16_f32", lambda: synth.rmat(20, 16, seed=0, dtype=np.float32), "f32c")],
    "uniform10k": [("uniform_10k_d1e-3", lambda: synth.uniform_random(10_000, 10_000, 1e-3, seed=0), "f64")],
    "rmat16": [("rmat_2e16_deg16", lambda: synth.rmat(16, 16, seed=0), "f64")],
    "rmat17": [("rmat_2e17_deg16", lambda: synth.rmat(17, 16, seed=0), "f64")],
}
WORKLOAD_DESC = {
    "lap2d1024+rmat20": "C=A*A for A = 2D 5-point Laplacian 1024^2 (FP64 4/-1) and A = R-MAT 2^20 "
                        "vertices, 16*2^20 edge samples, (a,b,c,d)=(.57,.19,.19,.05), FP64 U[0,1], seed 0",
    "rmat20_f32c": "C=A*A for A = R-MAT 2^20 vertices, degree 16, FP32 values U[0,1], seed 0; FP32 "
                   "compensated accumulation, rows over the error bound recomputed in FP64",
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _fp64_pipe(products: int, ms: float, sm_count: int, sm_mhz) -> dict:
    """The windowed numeric pass against GB300's FP64 pipe: every partial product costs two FP64
    operations there (the product a_ik * b_kj and the add inside the shared atomic), and the pipe
    executes 2 lanes per clock per SM (1.25 TFLOP/s counted as FMA), at the sampled SM clock."""
    mhz = float(sm_mhz) if sm_mhz else 2070.0
    peak = 2.0 * sm_count * mhz * 1e6
    achieved = 2.0 * products / (ms * 1e-3)
    return {"fp64_ops_per_s": round(achieved, 1), "fp64_peak_ops_per_s": round(peak, 1),
            "fp64_frac": round(achieved / peak, 4), "fp64_floor_ms": round(2.0 * products / peak * 1e3, 2)}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for r in csv.reader(f):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _traffic(kernel_file: str, workload: str, root: str = ROOT):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary, when it was
    taken on this workload with the kernel source as it is now (else None)."""
    import hashlib
    path = os.path.join(root, "profiles", f"k_num_window_{workload}.md")
    src = os.path.join(root, "paper_2004_13907_gb300", "csrc", kernel_file)
    try:
        want = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        fields = {}
        for line in open(path):
            # "- key: value" (the key may itself hold a colon, as in "sha256[:16]")
            m = re.match(r"\s*- (.+?): (.*)$", line)
            if m:
                fields[m.group(1).strip()] = m.group(2).strip().strip("`")
        if fields.get("kernel source sha256[:16]") != want:
            return None
        return int(fields["dram bytes per launch"].replace(",", ""))
    except Exception:
        return None


def _max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks, on every rank (a step is as slow as its slowest replica)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_gflops(products_per_rank: int, ranks: int, ms: float) -> float:
    """Whole-job GFLOP/s: every rank multiplies its own replica of the workload (2 flops per partial
    product) in the slowest rank's time."""
    return 2.0 * products_per_rank * ranks / (ms * 1e-3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _window_bytes(info: dict) -> tuple:
    """Algorithmic bytes of the windowed numeric pass (k_num_window, and k_expand_cols for the
    columns of rows whose bitmap the symbolic pass stored): per row 8 (its A row pointers), per
    A entry 12 (column, value) + 8 (start and end of the named B row), per partial product 12
    (the gathered B column and value), per entry of C 12 (column, value)."""
    rows = sum(info["num_class_rows"][0:4])
    annz = sum(info["num_class_annz"][0:4])
    prods = sum(info["num_class_products"][0:4])
    cnnz = sum(info["num_class_cnnz"][0:4])
    return 8 * rows + 20 * annz + 12 * prods + 12 * cnnz, prods


def _numeric_bytes(info: dict, m: int) -> int:
    """Algorithmic bytes of a whole numeric pass (all classes): A (row pointers, columns,
    values), the gathered B rows (row bounds, columns, values) and C (row pointers, columns,
    values)."""
    annz = sum(info["num_class_annz"])
    return 4 * (m + 1) + 12 * annz + 8 * annz + 12 * info["products"] + 8 * (m + 1) + 12 * info["nnz_c"]


def run_ours(args):
    import torch
    import paper_2004_13907_gb300 as sp

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    specs = WORKLOADS[args.workload]
    mats = [(name, gen()) for name, gen, _ in specs]
    precs = {name: prec for name, _, prec in specs}
    dev = [(name, M, sp.DeviceCSR.from_host(M, "cuda")) for name, M in mats]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    opts = sp.spgemm_opts_default(record_timings=1, fp64_accumulate=args.fp64_accumulate)
    stream = torch.cuda.current_stream()

    def step(collect=None):
        for name, M, dM in dev:
            plan = sp.spgemm_plan(dM, dM, precs[name], opts)
            sp.spgemm_symbolic(plan)
            C = sp.alloc_output(plan)
            sp.spgemm_numeric(plan, C)
            if collect is not None:
                collect.append((name, M, plan, C))
            else:
                del C
                sp.spgemm_plan_destroy(plan)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, per = [], {}
    launches = 0
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        col = []
        e0.record(stream)
        step(col)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for name, M, plan, C in col:
            sp.spgemm_plan_check(plan)
            info = sp.spgemm_plan_get_info(plan)
            tim = sp.spgemm_plan_get_timings(plan)
            launches += info["kernel_launches"]
            d = per.setdefault(name, {"info": info, "stages": {}, "rows": M.rows})
            for k, (ms, nl) in tim.items():
                d["stages"].setdefault(k, []).append(ms)
            sp.spgemm_plan_destroy(plan)
        del col
        C = plan = None    # drop the last product before the next step allocates its own
    wall = time.perf_counter() - t_wall0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()

    products_step = sum(per[n]["info"]["products"] for n, _, _ in dev)
    ms_local = float(np.mean(step_ms))
    ms = _max_over_ranks(ms_local, dist, "cuda")
    value = _job_gflops(products_step, ws, ms)

    # dominant kernel: the stage with the largest device time across the step (the windowed
    # numeric pass counts with the column expansion that completes its output)
    stage_tot = {}
    for name, d in per.items():
        for k, v in d["stages"].items():
            key = "num_window" if k == "num_expand" else k
            stage_tot[(name, key)] = stage_tot.get((name, key), 0.0) + float(np.mean(v))
    (dom_mat, dom_stage), dom_ms = max(stage_tot.items(), key=lambda kv: kv[1])
    peak, peak_kind = _peaks()
    roof = None
    if dom_stage == "num_window":
        bytes_, wprods = _window_bytes(per[dom_mat]["info"])
        achieved = bytes_ / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": f"k_num_window + k_expand_cols ({dom_mat})",
                "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes": bytes_,
                "launch_ms": round(dom_ms, 4), "traffic": _traffic("k_window.cu", args.workload)}
        if all(p == "f64" for p in precs.values()):
            roof.update(_fp64_pipe(wprods, dom_ms,
                                   torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count,
                                   clocks.get("sm_mhz")))
    breakdown = {}
    for name, d in per.items():
        info = d["info"]
        tot = sum(float(np.mean(v)) for v in d["stages"].values())
        breakdown[name] = {
            "rows": d["rows"], "products": info["products"], "nnz_c": info["nnz_c"],
            "stage_ms": {k: round(float(np.mean(v)), 4) for k, v in d["stages"].items() if np.mean(v) > 0},
            "kernel_ms_sum": round(tot, 4),
            "rows_redone_fp64": info["f32c_rerun_rows"],
            "numeric_ms": round(sum(float(np.mean(d["stages"][k])) for k in
                                    ("num_rowptr", "num_window", "num_expand", "num_block", "num_warp",
                                     "num_tiny")), 4),
            "numeric_alg_bytes": _numeric_bytes(info, d["rows"]),
            "num_class_rows": {sp._native.NUM_CLASSES[c]: info["num_class_rows"][c]
                               for c in range(len(sp._native.NUM_CLASSES)) if info["num_class_rows"][c]},
        }
        nb = breakdown[name]["numeric_alg_bytes"]
        breakdown[name]["numeric_GBps"] = round(nb / (breakdown[name]["numeric_ms"] * 1e-3) / 1e9, 1)
        breakdown[name]["numeric_frac_of_peak"] = round(breakdown[name]["numeric_GBps"] / peak, 4)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if all(p == "f64" for p in precs.values()) else "f32 (compensated) + f64 rerun",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOAD_DESC.get(args.workload, args.workload),
                   "products_per_step": products_step, "l2": "flushed: 512 MB written between timed steps",
                   "parallelism": f"replicas x{ws} (independent products, no collective on the data path)"},
        "roofline": roof, "gpu_launches": int(launches), "clocks": clocks,
        "breakdown": breakdown, "wall_s_timed": round(wall, 3),
    }
    # free the device-resident products before the end-to-end leg
    del dev
    torch.cuda.empty_cache()
    if not args.no_e2e:
        nnz_c = {name: per[name]["info"]["nnz_c"] for name, _ in mats}
        line["e2e"] = run_e2e(args, mats, nnz_c, products_step, sp, torch, dist)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mats, args.cpu_seconds)
    if dist:
        dist.destroy_process_group()
    return line, rank


def _batch_jobs(max_expected_products: float, limit: int = 4096):
    """Jobs of the batch distribution (n log-uniform in [100, 50000], density log-uniform in
    [1e-4, 1e-2]) whose expected product count n^3 d^2 is below the cap."""
    out = []
    for i in range(limit):
        n, d = synth.batch_job_params(i, 0)
        if n ** 3 * d * d < max_expected_products:
            out.append((i,) + synth.batch_job(i, 0))
    return out


def run_batch(args):
    """Batched form (one stacked product for every job) against the plain per-product launch
    (plan, symbolic, allocate, numeric per job), same jobs, same GPU."""
    import torch
    import paper_2004_13907_gb300 as sp
    cap = 1e6 if args.workload == "batch_small" else 1e7
    jobs = _batch_jobs(cap)
    dA = [sp.DeviceCSR.from_host(A, "cuda") for _, A, _ in jobs]
    dB = [sp.DeviceCSR.from_host(B, "cuda") for _, _, B in jobs]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    # autotuned bins: class thresholds and window merge cap chosen by timing this batch (untimed)
    tuned, tune_rep = sp.spgemm_autotune_batch(dA, dB, reps=2)

    def batched():
        b = sp.spgemm_batch(dA, dB, opts=tuned)
        return b

    def per_product():
        out = []
        for a, b in zip(dA, dB):
            out.append(sp.multiply(a, b))
        return out

    for _ in range(args.warmup):
        b = batched()
        b.destroy()
        per_product()
        flush.zero_()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    tb, tp, tr = [], [], []
    launches = 0
    products = 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b = batched()
        e1.record(stream)
        torch.cuda.synchronize()
        tb.append(e0.elapsed_time(e1))
        info = b.info()
        products = info["products"]
        launches += info["kernel_launches"]
        # numeric-only recompute through the captured graph
        b.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        b.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        tr.append(e0.elapsed_time(e1))
        b.destroy()
        flush.zero_()
        e0.record(stream)
        res = per_product()
        e1.record(stream)
        torch.cuda.synchronize()
        tp.append(e0.elapsed_time(e1))
        del res
    clocks = sampler.stop()
    ms_b, ms_p, ms_r = float(np.mean(tb)), float(np.mean(tp)), float(np.mean(tr))
    gf = lambda ms: round(2.0 * products / (ms * 1e-3) / 1e9, 3)
    return {
        "metric": METRIC, "value": gf(ms_b), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_b, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload,
                   "description": f"{len(jobs)} jobs of the batch distribution with expected products below "
                                  f"{cap:.0e} (n log-uniform [100, 50000], density log-uniform [1e-4, 1e-2], "
                                  f"A_j, B_j independent, FP64 U[-1,1], seed 0)",
                   "jobs": len(jobs), "products_per_step": products, "l2": "flushed between steps",
                   "parallelism": "one GPU, one stacked product"},
        "per_product_launch": {"value": gf(ms_p), "unit": UNIT, "ms_per_step": round(ms_p, 3),
                               "what": "plan + symbolic + allocate + numeric for each job in turn"},
        "batched_speedup": round(ms_p / ms_b, 2),
        "autotune": {"tiny_max": tuned.tiny_max, "warp_max": tuned.warp_max, "block_max": tuned.block_max,
                     "window_hash_fill": tuned.window_hash_fill, "trials": len(tune_rep["trials"]),
                     "default_ms": round(tune_rep["default_ms"], 3), "tuned_ms": round(tune_rep["best_ms"], 3)},
        "graph_replay": {"value": gf(ms_r), "unit": UNIT, "ms_per_step": round(ms_r, 4),
                         "what": "numeric-only recompute of every job as one CUDA graph launch"},
        "gpu_launches": int(launches), "clocks": clocks,
    }, 0


def _serve_job(kind: str, param: int):
    """Inputs of one served request (host CSR): A_i, B_i of the batch distribution, or a 3D
    7-point Laplacian A with B = A (None)."""
    if kind == "lap3d":
        return synth.laplacian3d(param), None
    return synth.batch_job(param, 0)


def _serve_inputs(reqs, procs: int):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        return pool.starmap(_serve_job, [(r.kind, r.param) for r in reqs], chunksize=2)


def _pct(v, q):
    """Nearest-rank percentile (the server's own definition)."""
    v = sorted(v)
    if not v:
        return 0.0
    k = int(np.ceil(q * len(v)))
    return float(v[max(k, 1) - 1])


def run_serve(args):
    """Serving: a Poisson stream of requests (90% jobs of the batch distribution, 10% A*A for a
    3D 7-point Laplacian with g in 64..128), FP64, 32 GB admission cap. The server (continuous
    batching) against the plain per-product launch (one product at a time, in arrival order):
    saturated throughput with every request queued at once, and p50/p99 latency (arrival to
    completion) at a Poisson rate of 0.8 x the plain path's saturated job throughput."""
    import threading
    import torch
    import paper_2004_13907_gb300 as sp
    R = args.serve_requests
    reqs = synth.serve_stream(R, 1.0, seed=0)
    t_gen = time.perf_counter()
    host = _serve_inputs(reqs, max(1, min(16, os.cpu_count() or 1)))
    t_gen = time.perf_counter() - t_gen
    dev = []
    for A, B in host:
        dA = sp.DeviceCSR.from_host(A, "cuda")
        dev.append((dA, dA if B is None else sp.DeviceCSR.from_host(B, "cuda")))
    torch.cuda.synchronize()
    in_bytes = sum(int(dA.col.numel()) * 12 + int(dB.col.numel()) * 12 for dA, dB in dev)
    del host
    cap = 32 << 30

    def server(**kw):
        if args.serve_small_products >= 0:
            kw["small_products"] = args.serve_small_products
        if args.serve_batch_entries > 0:
            kw["max_batch_entries"] = args.serve_batch_entries
        return sp.Server(mem_cap_bytes=cap, batch_window_us=args.serve_window_us, num_streams=args.serve_streams,
                         **kw)

    def drain(srv, ids, stall_s=600.0):
        """Consumes every result as it finishes (the server's completion queue), releasing each at
        once, as a client would; fails when no job has finished for stall_s seconds."""
        states = [None] * len(ids)
        pending = {i: k for k, i in enumerate(ids)}
        while pending:
            j = srv.wait_any(timeout=stall_s)
            if j is None:
                raise RuntimeError(f"serve: no job finished for {stall_s:.0f} s ({len(pending)} pending)")
            if j in pending:
                states[pending.pop(j)] = srv.poll(j)["state"]
                srv.release(j)
        return states

    # warm-up: the plain path and the server on the first requests
    for _ in range(args.warmup):
        for dA, dB in dev[:16]:
            sp.multiply(dA, dB)
        with server() as srv:
            drain(srv, [srv.submit(dA, dB, sync=False) for dA, dB in dev[:64]])
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    # saturated: every request queued at once
    sat = []
    rejected = set()
    for _ in range(args.steps):
        with server() as srv:
            ids = [srv.submit(dA, dB, sync=False) for dA, dB in dev]
            states = drain(srv, ids)
            st = srv.stats()
        rejected = {k for k, s_ in enumerate(states) if s_ != "done"}
        sat.append(st)
    products = sat[-1]["products"]
    ms_srv = float(np.mean([x["elapsed_s"] for x in sat])) * 1e3
    accepted = [k for k in range(R) if k not in rejected]
    plain_ms = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in accepted:
            C = sp.multiply(*dev[k])
            del C
        torch.cuda.synchronize()
        plain_ms.append((time.perf_counter() - t0) * 1e3)
    ms_plain = float(np.mean(plain_ms))
    # the rate of the latency runs comes from the plain path run the way it runs live (each
    # product waited for before the next), so that its queue is stable at 0.8 of capacity
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in accepted:
        C = sp.multiply(*dev[k])
        torch.cuda.synchronize()
        del C
    ms_plain_sync = (time.perf_counter() - t0) * 1e3
    lam = 0.8 * len(accepted) / (ms_plain_sync * 1e-3)
    arrival = np.array([r.arrival_s for r in reqs]) / lam
    # plain path at rate lam: each request runs when it has arrived and the previous one is done
    lat_plain = []
    t0 = time.perf_counter()
    for k in accepted:
        wait = t0 + arrival[k] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        C = sp.multiply(*dev[k])
        torch.cuda.synchronize()
        lat_plain.append((time.perf_counter() - t0 - arrival[k]) * 1e3)
        del C
    # server at rate lam: a submitter thread follows the arrival times, this thread consumes
    with server() as srv:
        lag = [0.0]
        ready = threading.Event()

        def submitter():
            t0s = time.perf_counter()
            ready.set()
            for k in range(R):
                wait = t0s + arrival[k] - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                lag[0] = max(lag[0], time.perf_counter() - t0s - arrival[k])
                srv.submit(*dev[k], sync=False)
        th = threading.Thread(target=submitter)
        th.start()
        ready.wait()
        for _ in range(R):   # every request finishes once; each result is released as it comes out
            j = srv.wait_any(timeout=600.0)
            if j is None:
                raise RuntimeError("serve: no job finished for 600 s")
            srv.release(j)
        th.join()
        live = srv.stats()
    clocks = sampler.stop()
    gf = lambda p, ms: round(2.0 * p / (ms * 1e-3) / 1e9, 3)
    n_lap = sum(1 for r in reqs if r.kind == "lap3d")
    return {
        "metric": METRIC, "value": gf(products, ms_srv), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_srv, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serve",
                   "description": f"{R} requests of a Poisson stream (seed 0): {R - n_lap} jobs A_i*B_i of the "
                                  f"batch distribution (n log-uniform [100, 50000], density log-uniform "
                                  f"[1e-4, 1e-2]), {n_lap} A*A for 3D 7-point Laplacians with g in 64..128; "
                                  f"FP64; 32 GB admission cap; inputs resident on the device",
                   "requests": R, "input_bytes": in_bytes, "products_per_step": products,
                   "l2": "inputs larger than L2",
                   "parallelism": f"one GPU, continuous batching, {args.serve_streams} streams",
                   "batch_window_us": args.serve_window_us, "input_generation_s": round(t_gen, 1)},
        "saturated": {"server_ms": round(ms_srv, 3), "plain_ms": round(ms_plain, 3),
                      "plain_value": gf(products, ms_plain), "speedup": round(ms_plain / ms_srv, 3),
                      "server_jobs_per_s": round(sat[-1]["jobs_per_s"], 1),
                      "mean_batch_jobs": round(sat[-1]["mean_batch_jobs"], 2),
                      "rejected_over_cap": len(rejected), "splits": sat[-1]["splits"],
                      "bytes_peak": sat[-1]["bytes_peak"]},
        "latency": {"rate_per_s": round(lam, 2), "what": "arrival to completion, ms, at 0.8 x the job rate "
                                                          "of the plain path run one product at a time",
                    "plain_capacity_ms": round(ms_plain_sync, 3),
                    "server_p50_ms": round(live["latency_p50_ms"], 3), "server_p99_ms": round(live["latency_p99_ms"], 3),
                    "server_max_ms": round(live["latency_max_ms"], 3),
                    "plain_p50_ms": round(_pct(lat_plain, 0.5), 3), "plain_p99_ms": round(_pct(lat_plain, 0.99), 3),
                    "plain_max_ms": round(max(lat_plain), 3),
                    "server_mean_batch_jobs": round(live["mean_batch_jobs"], 2),
                    "submit_lag_max_ms": round(lag[0] * 1e3, 3)},
        "gpu_launches": int(sat[-1]["kernel_launches"]), "clocks": clocks,
    }, 0


def _pinned(n: int, dtype, torch):
    """Page-locked host array of exactly n elements (numpy memory registered with CUDA)."""
    a = np.empty(max(n, 1), dtype=dtype)
    t = torch.from_numpy(a)
    rc = torch.cuda.cudart().cudaHostRegister(t.data_ptr(), t.numel() * t.element_size(), 0)
    return t, (int(rc) == 0)


def run_e2e(args, mats, nnz_c, products_step, sp, torch, dist):
    """Same metric through spgemm_multiply_host: host A -> device, product, C -> host.
    Host arrays are page-locked; the output arrays are sized from nnz(C) of the device run."""
    hosts = []
    pinned_ok = True
    for name, M in mats:
        rp, ok1 = _pinned(M.rows + 1, np.int32, torch)
        col, ok2 = _pinned(M.nnz, np.int32, torch)
        val, ok3 = _pinned(M.nnz, np.float64, torch)
        rp.copy_(torch.from_numpy(M.row_ptr.astype(np.int32)))
        col[:M.nnz].copy_(torch.from_numpy(M.col))
        val[:M.nnz].copy_(torch.from_numpy(M.val))
        hA = sp.DeviceCSR(M.rows, M.cols, rp, col[:M.nnz], val[:M.nnz])
        nnz = nnz_c[name]
        idx64 = nnz >= 2**31
        orp, o1 = _pinned(M.rows + 1, np.int64 if idx64 else np.int32, torch)
        ocol, o2 = _pinned(nnz, np.int32, torch)
        oval, o3 = _pinned(nnz, np.float64, torch)
        pinned_ok &= all((ok1, ok2, ok3, o1, o2, o3))
        out = sp.DeviceCSR(M.rows, M.cols, orp, ocol[:nnz], oval[:nnz])
        h2d = 2 * ((M.rows + 1) * 4 + M.nnz * 12)            # A and B (= A) copied in
        d2h = (M.rows + 1) * orp.element_size() + nnz * 12    # C copied out
        hosts.append((name, hA, out, idx64, h2d, d2h))

    per_matrix = {name: [] for name, *_ in hosts}

    def step():
        for name, hA, out, idx64, _, _ in hosts:
            t = time.perf_counter()
            sp.spgemm_multiply_host(hA, hA, out=out, idx64=idx64)
            per_matrix[name].append(time.perf_counter() - t)

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    for v in per_matrix.values():
        v.clear()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    ws, _, _ = _dist()
    t = _max_over_ranks(float(np.mean(times)), dist, "cuda")
    return {"value": round(_job_gflops(products_step, ws, t * 1e3), 3), "unit": UNIT,
            "h2d_bytes_per_step": int(sum(h[4] for h in hosts)),
            "d2h_bytes_per_step": int(sum(h[5] for h in hosts)),
            "ms_per_step": round(t * 1e3, 3), "host_buffers": "pinned" if pinned_ok else "pageable (pinning failed)",
            "ms_per_matrix": {k: round(float(np.mean(v)) * 1e3, 3) for k, v in per_matrix.items()},
            "api": "spgemm_multiply_host (C ABI, host buffers)"}


def cpu_baseline(mats, seconds: float) -> dict:
    """The CPU oracle (ordered-map Gustavson, threaded over rows) on a seeded row sample of
    each matrix sized to about ``seconds`` of work, extrapolated to the workload."""
    import oracle
    total_t = 0.0
    total_p = 0
    samples = []
    threads = 0
    for name, M in mats:
        P = oracle.products_per_row(M, M)
        rate_probe = 3e7  # products/s guess used only to size the sample
        budget = max(int(seconds / len(mats) * rate_probe), 1)
        if P.sum() <= budget:
            rows = None
            sampled = int(P.sum())
        else:
            rng = np.random.default_rng(1234)
            order = rng.permutation(M.rows)
            cs = np.cumsum(P[order])
            k = int(np.searchsorted(cs, budget)) + 1
            rows = np.sort(order[:k])
            sampled = int(P[rows].sum())
        t0 = time.perf_counter()
        out = oracle.spgemm(M, M, rows=rows)
        dt = time.perf_counter() - t0
        threads = max(threads, out.threads)
        rate = sampled / dt
        total_t += int(P.sum()) / rate
        total_p += int(P.sum())
        samples.append(f"{name}: {'all' if rows is None else len(rows)} rows, {sampled} products in {dt:.2f} s")
    return {"value": round(2.0 * total_p / total_t / 1e9, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "; ".join(samples) + " (time extrapolated to the whole workload by products)"}


def run_reference(args):
    """The CPU oracle as the reference arm: each step multiplies a bounded seeded row sample
    of every matrix of the workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return None, rank
    import oracle
    mats = [(name, gen()) for name, gen, _ in WORKLOADS[args.workload]]
    Ps = [oracle.products_per_row(M, M) for _, M in mats]
    budget = int(args.ref_products_per_step)
    rng = np.random.default_rng(99)
    rows_per = []
    for (name, M), P in zip(mats, Ps):
        b = budget // len(mats)
        order = rng.permutation(M.rows)
        cs = np.cumsum(P[order])
        k = int(np.searchsorted(cs, b)) + 1
        rows_per.append(np.sort(order[:min(k, M.rows)]))

    def step():
        prods = 0
        threads = 0
        for (name, M), P, rows in zip(mats, Ps, rows_per):
            out = oracle.spgemm(M, M, rows=rows)
            threads = max(threads, out.threads)
            prods += int(P[rows].sum())
        return prods, threads

    for _ in range(args.warmup):
        step()
    times, prods, threads = [], 0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        p, threads = step()
        times.append(time.perf_counter() - t0)
        prods = p
    t = float(np.mean(times))
    value = 2.0 * prods / t / 1e9
    sample = "; ".join(f"{name}: {len(r)} seeded random rows" for (name, _), r in zip(mats, rows_per))
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOAD_DESC.get(args.workload, args.workload),
                   "products_per_step": prods, "l2": "n/a (CPU)", "parallelism": "host threads"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample + f" per step ({prods} products)"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line, rank


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lap2d1024+rmat20",
                    choices=sorted(WORKLOADS) + ["batch_small", "batch_mid", "serve"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-accumulate", type=int, default=0, choices=[0, 1, 2],
                    help="FP64 sums: 0 shared atomics (default), 1 exact fixed point on the windowed rows, "
                         "2 deterministic (every row windowed, exact)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-products-per-step", type=float, default=2e8)
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--serve-requests", type=int, default=600)
    ap.add_argument("--serve-window-us", type=int, default=300)
    ap.add_argument("--serve-streams", type=int, default=2)
    ap.add_argument("--serve-small-products", type=int, default=-1, help="server default when negative")
    ap.add_argument("--serve-batch-entries", type=int, default=0, help="server default when 0")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        sys.stderr.write("note: fewer than 3 warm-up steps\n")
    if args.impl == "reference":
        line, rank = run_reference(args)
    elif args.workload.startswith("batch"):
        line, rank = run_batch(args)
    elif args.workload == "serve":
        line, rank = run_serve(args)
    else:
        line, rank = run_ours(args)
    if rank == 0 and line is not None:
        s = json.dumps(line)
        print(s, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(s + "\n")


if __name__ == "__main__":
    main()
