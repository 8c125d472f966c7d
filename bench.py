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
    "rmat17_f32c": [("rmat_2e17_deg16_f32", lambda: synth.rmat(17, 16, seed=0, dtype=np.float32), "f32c")],
}
DEFAULT_WORKLOAD = "lap2d1024+rmat20"
WORKLOAD_DESC = {
    "lap2d1024+rmat20": "C=A*A for A = 2D 5-point Laplacian 1024^2 (FP64 4/-1) and A = R-MAT 2^20 "
                        "vertices, 16*2^20 edge samples, (a,b,c,d)=(.57,.19,.19,.05), FP64 U[0,1], seed 0",
    "rmat20_f32c": "C=A*A for A = R-MAT 2^20 vertices, degree 16, FP32 values U[0,1], seed 0; FP32 "
                   "compensated accumulation, rows over the error bound recomputed in FP64",
    "uniform10k": "C=A*A for A 10,000 x 10,000, Binomial(n, 1e-3) distinct uniform columns per row, FP64 "
                  "U[-1,1), seed 0",
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


def _traffic(alg_bytes: int, root: str = ROOT):
    """DRAM bytes of the windowed pass (k_num_window + k_expand_cols) per launch: the committed
    small-case record (R-MAT 2^17, one-pass ncu launch list) gives DRAM bytes per algorithmic byte,
    scaled to this launch by its algorithmic bytes; None when the record was taken on another
    version of the kernel source."""
    import hashlib
    path = os.path.join(root, "profiles", "k_num_window_rmat17.md")
    src = os.path.join(root, "paper_2004_13907_gb300", "csrc", "k_window.cu")
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
        return int(round(float(fields["dram bytes per algorithmic byte"]) * alg_bytes))
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


def _window_bytes(info: dict, vbytes: int = 8) -> tuple:
    """Algorithmic bytes of the windowed numeric pass (k_num_window, and k_expand_cols for the
    columns of rows whose bitmap the symbolic pass stored): per row 8 (its A row pointers), per
    A entry 4 + v (column, value) + 8 (start and end of the named B row), per partial product
    4 + v (the gathered B column and value), per entry of C 4 + v (column, value); v = 8 (FP64)
    or 4 (FP32)."""
    rows = sum(info["num_class_rows"][0:4])
    annz = sum(info["num_class_annz"][0:4])
    prods = sum(info["num_class_products"][0:4])
    cnnz = sum(info["num_class_cnnz"][0:4])
    return 8 * rows + (12 + vbytes) * annz + (4 + vbytes) * prods + (4 + vbytes) * cnnz, prods


def _vbytes(prec: str) -> int:
    return 4 if prec == "f32c" else 8


def _class_bytes(info: dict, vbytes: int = 8) -> dict:
    """Algorithmic bytes of each numeric row class's kernel: per row 8 (its A row pointers) + 8
    (its C row pointer), per A entry 4 + v (column, value) + 8 (start and end of the named B row),
    per partial product 4 + v (the gathered B column and value), per entry of C 4 + v."""
    import paper_2004_13907_gb300 as sp
    out = {}
    for c, name in enumerate(sp._native.NUM_CLASSES):
        rows = info["num_class_rows"][c]
        if rows and name != "empty":
            out[name] = (16 * rows + (12 + vbytes) * info["num_class_annz"][c] +
                         (4 + vbytes) * info["num_class_products"][c] + (4 + vbytes) * info["num_class_cnnz"][c])
    return out


def _numeric_bytes(info: dict, m: int, vbytes: int = 8) -> int:
    """Algorithmic bytes of a whole numeric pass (all classes): A (row pointers, columns,
    values), the gathered B rows (row bounds, columns, values) and C (row pointers, columns,
    values); v = 8 (FP64) or 4 (FP32) bytes per value."""
    annz = sum(info["num_class_annz"])
    return (4 * (m + 1) + (4 + vbytes) * annz + 8 * annz + (4 + vbytes) * info["products"] + 8 * (m + 1) +
            (4 + vbytes) * info["nnz_c"])


def _product_config(wl: str, args, sp, torch, steps: int, warmup: int, cpu_err: bool = False) -> dict:
    """One plain product workload (C = A*A per matrix, all timed together), as the headline line
    times it; the roofline of its dominant stage. With cpu_err, the CPU-baseline leg (the oracle
    on a bounded row sample) also gives the product's max relative entry error on that sample."""
    specs = WORKLOADS[wl]
    mats = [(name, gen()) for name, gen, _ in specs]
    precs = {name: prec for name, _, prec in specs}
    dev = [(name, M, sp.DeviceCSR.from_host(M, "cuda")) for name, M in mats]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    # the timed steps run the product as a caller does (default options); the stage breakdown
    # comes from as many steps again with stage events, which cost microseconds per plan (a tenth
    # of a small product)
    opts = sp.spgemm_opts_default()
    opts_staged = sp.spgemm_opts_default(record_timings=1)
    stream = torch.cuda.current_stream()
    peak, _ = _peaks()

    def step(o):
        out = []
        for name, M, dM in dev:
            plan = sp.spgemm_plan(dM, dM, precs[name], o)
            sp.spgemm_symbolic(plan)
            C = sp.alloc_output(plan)
            sp.spgemm_numeric(plan, C)
            out.append((name, plan, C))
        return out

    for _ in range(warmup):
        for name, plan, C in step(opts):
            sp.spgemm_plan_destroy(plan)
        flush.zero_()
    torch.cuda.synchronize()
    times, stages, products, launches, infos = [], {}, 0, 0, {}
    for staged in (False, True):
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = step(opts_staged if staged else opts)
            e1.record(stream)
            torch.cuda.synchronize()
            if not staged:
                times.append(e0.elapsed_time(e1))
            products = 0
            for name, plan, C in res:
                sp.spgemm_plan_check(plan)
                info = sp.spgemm_plan_get_info(plan)
                infos[name] = info
                products += info["products"]
                if not staged:
                    launches += info["kernel_launches"]
                else:
                    step_st = {}
                    for k, (ms, _) in sp.spgemm_plan_get_timings(plan).items():
                        key = (name, "num_window" if k == "num_expand" else k)   # the expansion completes the pass
                        step_st[key] = step_st.get(key, 0.0) + ms
                    for key, ms in step_st.items():
                        stages.setdefault(key, []).append(ms)
                sp.spgemm_plan_destroy(plan)
            del res
    ms = float(np.mean(times))
    st = {k: float(np.mean(v)) for k, v in stages.items()}
    (dom_name, dom_stage), dom_ms = max(st.items(), key=lambda kv: kv[1])
    name0, M0, _ = dev[0]
    numeric_ms = sum(v for (n_, k), v in st.items() if k.startswith("num_"))
    nbytes = sum(_numeric_bytes(infos[n], M.rows, _vbytes(precs[n])) for n, M, _ in dev)
    out = {"workload": wl, "value": round(_job_gflops(products, 1, ms), 3), "unit": UNIT, "ms_per_step": round(ms, 4),
           "steps": steps, "warmup": warmup, "products_per_step": products, "gpu_launches": int(launches),
           "description": WORKLOAD_DESC.get(wl, wl),
           "numeric": {"ms": round(numeric_ms, 4), "alg_bytes": nbytes,
                       "GBps": round(nbytes / (numeric_ms * 1e-3) / 1e9, 1),
                       "frac_of_peak": round(nbytes / (numeric_ms * 1e-3) / 1e9 / peak, 4)},
           "stage_ms": {f"{n}:{k}": round(v, 4) for (n, k), v in st.items() if v > 0.001},
           "stage_timing": "stage events in as many further steps (the timed steps run default options)"}
    if dom_stage == "num_window":
        wb, _ = _window_bytes(infos[dom_name], _vbytes(precs[dom_name]))
        out["roofline"] = {"bound": "hbm", "kernel": f"k_num_window + k_expand_cols ({dom_name})",
                           "achieved": round(wb / (dom_ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(wb / (dom_ms * 1e-3) / 1e9 / peak, 4), "algorithmic_bytes": wb,
                           "launch_ms": round(dom_ms, 4)}
    if any(p_ == "f32c" for p_ in precs.values()):
        out["rows_redone_fp64"] = int(sum(i["f32c_rerun_rows"] for i in infos.values()))
    if cpu_err:
        # CPU-baseline leg: the oracle on a bounded row sample of the product, its rate, and the
        # GPU result's error on those rows (FP32 results against the FP64 oracle)
        res = step(opts)
        torch.cuda.synchronize()
        out["cpu_baseline"], out["max_rel_err"] = cpu_baseline_error(mats, res, args.cpu_seconds, sp)
        for name, plan, C in res:
            sp.spgemm_plan_destroy(plan)
        del res
    del dev, flush
    torch.cuda.empty_cache()
    return out


def config_reuse(args, sp, torch, steps: int, warmup: int) -> dict:
    """Plan reuse (the symbolic/numeric split): numeric-only recompute on an existing plan, with
    the input values changed in place between steps (same pattern), against the whole product
    (plan, symbolic, allocate, numeric), FP64; on the 2D Laplacian 1024^2 and R-MAT 2^20 squares,
    and on the multigrid Galerkin coarse operator R*(A*P) of the Laplacian (2x2 aggregation, two
    products, the second reading the first's output)."""
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def ev_time(fn):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    def chain(stages):
        """stages: list of (A, B-or-index of an earlier stage's output); returns [(plan, C)]"""
        out = []
        for A, B in stages:
            Bm = out[B][1] if isinstance(B, int) else B
            plan = sp.spgemm_plan(A, Bm)
            sp.spgemm_symbolic(plan)
            C = sp.alloc_output(plan)
            sp.spgemm_numeric(plan, C)
            out.append((plan, C))
        return out

    def destroy(res):
        for plan, _ in res:
            sp.spgemm_plan_destroy(plan)

    cases = {}
    L = synth.laplacian2d(1024)
    dL = sp.DeviceCSR.from_host(L, "cuda")
    cases["lap2d1024"] = (dL, [(dL, dL)])
    Rm = synth.rmat(20, 16, seed=0)
    dRm = sp.DeviceCSR.from_host(Rm, "cuda")
    cases["rmat20"] = (dRm, [(dRm, dRm)])
    dP = sp.DeviceCSR.from_host(synth.aggregation_prolongator(1024), "cuda")
    dR = sp.DeviceCSR.from_host(synth.aggregation_restrictor(1024), "cuda")
    cases["galerkin_lap2d1024"] = (dL, [(dL, dP), (dR, 0)])
    out = {}
    for name, (dA, stages) in cases.items():
        for _ in range(warmup):
            destroy(chain(stages))
        full = []
        products = 0
        for _ in range(steps):
            ms, res = ev_time(lambda: chain(stages))
            full.append(ms)
            products = sum(sp.spgemm_plan_get_info(p)["products"] for p, _ in res)
            destroy(res)
        res = chain(stages)
        torch.cuda.synchronize()

        def numeric_only():
            for plan, C in res:
                sp.spgemm_numeric(plan, C)

        for _ in range(warmup):
            dA.val.mul_(1.0 + 2.0 ** -20)
            numeric_only()
        num = []
        for _ in range(steps):
            dA.val.mul_(1.0 + 2.0 ** -20)   # new values, same pattern (outside the timed region)
            ms, _ = ev_time(numeric_only)
            num.append(ms)
        for plan, _ in res:
            sp.spgemm_plan_check(plan)
        destroy(res)
        del res
        ms_f, ms_n = float(np.mean(full)), float(np.mean(num))
        out[name] = {"products": products, "full_ms": round(ms_f, 4), "numeric_only_ms": round(ms_n, 4),
                     "full_value": round(2.0 * products / (ms_f * 1e-3) / 1e9, 3),
                     "numeric_only_value": round(2.0 * products / (ms_n * 1e-3) / 1e9, 3),
                     "speedup": round(ms_f / ms_n, 3), "unit": UNIT, "steps": steps, "warmup": warmup}
    out["description"] = ("numeric-only recompute on an existing plan (input values changed in place between steps) "
                          "against the whole product; Galerkin R*(A*P) with 2x2 aggregation of the 1024^2 Laplacian "
                          "(coarse operator = 2 x the 512^2 Laplacian, checked in the tests)")
    del cases, dL, dRm, dP, dR, flush
    torch.cuda.empty_cache()
    return out


def run_one_config(args):
    """One of the other configurations alone (printed as its own JSON line)."""
    import torch
    import paper_2004_13907_gb300 as sp
    torch.cuda.set_device(0)
    sw, ss = max(3, args.side_warmup), max(1, args.side_steps)
    name = args.config
    if name == "uniform10k":
        return _product_config("uniform10k", args, sp, torch, max(ss, 10), max(sw, 10)), 0
    if name == "plan_reuse":
        return config_reuse(args, sp, torch, max(ss, 5), sw), 0
    if name == "rmat20_f32c":
        return _product_config("rmat20_f32c", args, sp, torch, ss, sw, cpu_err=True), 0
    if name == "batch4096":
        return config_batch(args, sp, torch, _device_jobs(range(BATCH_JOBS), sp, torch), sw, 1), 0
    return config_serve(args, sp, torch, _device_jobs(range(SERVE_POOL), sp, torch), args.serve_requests, sw), 0


def run_configs(args, sp, torch) -> dict:
    """The other measured configurations, each as its own object: the uniform 10k product, the
    R-MAT 2^20 FP32-compensated product (with its max relative error against the FP64 oracle),
    the full 4,096-job batch against per-product launches, and the 20,000-request serving
    stream against the plain path."""
    out = {}
    sw, ss = max(3, args.side_warmup), max(1, args.side_steps)
    t0 = time.perf_counter()
    out["uniform10k"] = _product_config("uniform10k", args, sp, torch, max(ss, 10), max(sw, 10))
    out["plan_reuse"] = config_reuse(args, sp, torch, max(ss, 5), sw)
    out["rmat20_f32c"] = _product_config("rmat20_f32c", args, sp, torch, ss, sw, cpu_err=True)
    jobs = _device_jobs(range(BATCH_JOBS), sp, torch)
    out["batch4096"] = config_batch(args, sp, torch, jobs, sw, 1)
    for i in list(jobs):
        if i >= SERVE_POOL:
            del jobs[i]
    torch.cuda.empty_cache()
    out["serve20000"] = config_serve(args, sp, torch, jobs, args.serve_requests, sw)
    del jobs
    torch.cuda.empty_cache()
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


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
        bytes_, wprods = _window_bytes(per[dom_mat]["info"], _vbytes(precs[dom_mat]))
        achieved = bytes_ / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": f"k_num_window + k_expand_cols ({dom_mat})",
                "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes": bytes_,
                "launch_ms": round(dom_ms, 4), "traffic": None, "traffic_source": None}
        if all(p == "f64" for p in precs.values()):
            roof["traffic"] = _traffic(bytes_)
            roof["traffic_source"] = ("R-MAT 2^17 DRAM bytes per algorithmic byte (profiles/k_num_window_rmat17.md) x "
                                      "this launch's algorithmic bytes; B fits L2 at 2^17, so a lower bound here")
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
            "numeric_alg_bytes": _numeric_bytes(info, d["rows"], _vbytes(precs[name])),
            "num_class_rows": {sp._native.NUM_CLASSES[c]: info["num_class_rows"][c]
                               for c in range(len(sp._native.NUM_CLASSES)) if info["num_class_rows"][c]},
            "num_class_alg_bytes": _class_bytes(info, 4 if precs[name] == "f32c" else 8),
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
    if ws == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_configs:
        line["configs"] = run_configs(args, sp, torch)
    if dist:
        dist.destroy_process_group()
    return line, rank


BATCH_JOBS = 4096          # jobs of the batching config
SERVE_REQUESTS = 20_000    # requests of the serving config
SERVE_POOL = 512           # distinct batch-distribution jobs the served requests draw from
WAVE_OUT_BYTES = 48 << 30  # estimated output bytes per batched wave (outputs are freed per wave)


def _job_estimate(i: int) -> tuple:
    """(n, d, expected partial products n^3 d^2, expected nnz(C) n^2 (1 - exp(-n d^2))) of job i."""
    import math
    n, d = synth.batch_job_params(i, 0)
    return n, d, n ** 3 * d * d, n * n * (1.0 - math.exp(-n * d * d))


def _device_jobs(idx, sp, torch) -> dict:
    """Jobs of the batch distribution built in device memory by synth.torch_gen (bit-identical to
    synth.batch_job, which the tests and the oracle use)."""
    from synth import torch_gen
    out = {}
    for i in idx:
        n, (arp, acol, aval), (brp, bcol, bval) = torch_gen.batch_job(i, 0, device="cuda")
        out[i] = (sp.DeviceCSR(n, n, arp, acol, aval), sp.DeviceCSR(n, n, brp, bcol, bval))
    torch.cuda.synchronize()
    return out


def _waves(idx, cap_bytes: float) -> list:
    """Consecutive jobs grouped while their estimated outputs (12 bytes per entry) stay within
    cap_bytes; a job larger than the cap is a wave of its own."""
    waves, cur, acc = [], [], 0.0
    for i in idx:
        b = 12.0 * _job_estimate(i)[3] + 8.0 * _job_estimate(i)[0]
        if cur and acc + b > cap_bytes:
            waves.append(cur)
            cur, acc = [], 0.0
        cur.append(i)
        acc += b
    if cur:
        waves.append(cur)
    return waves


def config_batch(args, sp, torch, jobs: dict, warmup: int, steps: int) -> dict:
    """Batching (4,096 independent products A_j*B_j of the batch distribution): the batched form
    against the plain per-product launch (plan, symbolic, allocate, numeric for each job in
    turn), same jobs, same GPU, FP64. The batched form groups the jobs by size: the small-job
    stratum (expected P < 1e6, where launch overhead is what batching removes) and the larger
    jobs, each stratum in waves of one stacked product whose outputs fit WAVE_OUT_BYTES (every
    output freed before the next wave), each stratum with its own autotuned bins (tuned on the
    small stratum, and on a sample of large jobs). The small stratum is also reported alone,
    with its CUDA-graph numeric replay."""
    stream = torch.cuda.current_stream()
    idx = sorted(jobs)
    small = [i for i in idx if _job_estimate(i)[2] < 1e6]
    large = [i for i in idx if _job_estimate(i)[2] >= 1e6]
    sA = [jobs[i][0] for i in small]
    sB = [jobs[i][1] for i in small]
    tuned, tune_rep = sp.spgemm_autotune_batch(sA, sB, reps=2)
    sample = [i for i in large if 1e7 <= _job_estimate(i)[2] <= 3e8][:48]
    tuned_l, tune_rep_l = sp.spgemm_autotune_batch([jobs[i][0] for i in sample], [jobs[i][1] for i in sample],
                                                   reps=2)
    waves = [(w, tuned) for w in _waves(small, WAVE_OUT_BYTES)] + \
            [(w, tuned_l) for w in _waves(large, WAVE_OUT_BYTES)]

    def batched(ids_waves):
        prods = 0
        launches = 0
        for w, o in ids_waves:
            b = sp.spgemm_batch([jobs[i][0] for i in w], [jobs[i][1] for i in w], opts=o)
            info = b.info()
            prods += info["products"]
            launches += info["kernel_launches"]
            b.destroy()
        return prods, launches

    def plain(ids):
        for i in ids:
            C = sp.multiply(jobs[i][0], jobs[i][1])
            del C

    def timed(fn, *a):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn(*a)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    # warm-up: one whole pass of each form (allocator pools reach their high-water mark), then
    # the small stratum
    for wu in range(warmup):
        if wu == 0:
            batched(waves)
            plain(idx)
            torch.cuda.empty_cache()
        else:
            batched([(small, tuned)])
            plain(small)
    tb, tp, ts_b, ts_p, tr = [], [], [], [], []
    products = launches = small_products = 0
    for _ in range(steps):
        ms, (products, launches) = timed(batched, waves)
        tb.append(ms)
        ms, _ = timed(plain, idx)
        tp.append(ms)
        torch.cuda.empty_cache()
        ms, (small_products, _) = timed(batched, [(small, tuned)])
        ts_b.append(ms)
        ms, _ = timed(plain, small)
        ts_p.append(ms)
        b = sp.spgemm_batch(sA, sB, opts=tuned)
        b.replay()
        torch.cuda.synchronize()
        ms, _ = timed(b.replay)
        tr.append(ms)
        b.destroy()
    gf = lambda p, ms: round(2.0 * p / (ms * 1e-3) / 1e9, 3)
    ms_b, ms_p = float(np.mean(tb)), float(np.mean(tp))
    return {
        "workload": f"batch{len(idx)}", "value": gf(products, ms_b), "unit": UNIT, "ms_per_step": round(ms_b, 3),
        "steps": steps, "warmup": warmup, "jobs": len(idx), "waves": len(waves), "products_per_step": products,
        "plain_value": gf(products, ms_p), "plain_ms_per_step": round(ms_p, 3),
        "speedup_vs_plain": round(ms_p / ms_b, 3), "gpu_launches": int(launches),
        "small_stratum": {"jobs": len(small), "products": small_products,
                          "value": gf(small_products, float(np.mean(ts_b))),
                          "plain_value": gf(small_products, float(np.mean(ts_p))),
                          "speedup_vs_plain": round(float(np.mean(ts_p)) / float(np.mean(ts_b)), 3),
                          "graph_replay_value": gf(small_products, float(np.mean(tr)))},
        "autotune": {"small": {"tiny_max": tuned.tiny_max, "warp_max": tuned.warp_max, "block_max": tuned.block_max,
                               "window_hash_fill": tuned.window_hash_fill, "trials": len(tune_rep["trials"]),
                               "tuned_on": f"{len(small)} jobs with expected P < 1e6"},
                     "large": {"tiny_max": tuned_l.tiny_max, "warp_max": tuned_l.warp_max,
                               "block_max": tuned_l.block_max, "window_hash_fill": tuned_l.window_hash_fill,
                               "trials": len(tune_rep_l["trials"]),
                               "tuned_on": f"{len(sample)} jobs with expected P in [1e7, 3e8]"}},
        "description": f"{len(idx)} jobs C_j = A_j*B_j, n log-uniform [100, 50000], density log-uniform "
                       f"[1e-4, 1e-2], A_j, B_j independent, FP64 U[-1,1), seed 0; batched form in {len(waves)} "
                       f"waves (small-job stratum, then larger jobs) of at most {WAVE_OUT_BYTES >> 30} GiB of "
                       f"expected output, each output freed before the next wave; warm-up: one whole pass of "
                       f"each form, then the small stratum",
    }


def _pct(v, q):
    """Nearest-rank percentile (the server's own definition)."""
    v = sorted(v)
    if not v:
        return 0.0
    k = int(np.ceil(q * len(v)))
    return float(v[max(k, 1) - 1])


def config_serve(args, sp, torch, jobs: dict, requests: int, warmup: int) -> dict:
    """Serving: a Poisson stream of `requests` requests (90% jobs of the batch distribution, 10%
    A*A for a 3D 7-point Laplacian with g in 64..128), FP64, 32 GB admission cap. Request i of
    the batch kind takes job (i mod SERVE_POOL) of the batch distribution; the Laplacians are built
    once per grid size. The server (continuous batching) against the plain per-product launch
    (one product at a time, in arrival order): saturated throughput (every request queued at
    once for the server, one after the other for the plain path), and p50/p99 latency (arrival
    to completion) at a Poisson rate of 0.8 x the plain path's job rate."""
    import threading
    R = requests
    reqs = synth.serve_stream(R, 1.0, seed=0)
    lap = {}
    for r in reqs:
        if r.kind == "lap3d" and r.param not in lap:
            L = sp.DeviceCSR.from_host(synth.laplacian3d(r.param), "cuda")
            lap[r.param] = (L, L)
    dev = [lap[r.param] if r.kind == "lap3d" else jobs[r.index % SERVE_POOL] for r in reqs]
    torch.cuda.synchronize()
    cap = 32 << 30

    def server(**kw):
        return sp.Server(mem_cap_bytes=cap, batch_window_us=args.serve_window_us, num_streams=args.serve_streams,
                         **kw)

    def drain(srv, n, stall_s=600.0):
        """Takes every result from the server's completion queue as it finishes, releasing each
        at once, as a client would."""
        states = {}
        for _ in range(n):
            j = srv.wait_any(timeout=stall_s)
            if j is None:
                raise RuntimeError(f"serve: no job finished for {stall_s:.0f} s")
            states[j] = srv.poll(j)["state"]
            srv.release(j)
        return states

    for _ in range(warmup):
        for dA, dB in dev[:16]:
            sp.multiply(dA, dB)
        with server() as srv:
            for dA, dB in dev[:200]:
                srv.submit(dA, dB, sync=False)
            drain(srv, 200)
    torch.cuda.synchronize()
    # saturated server: every request queued at once
    with server() as srv:
        ids = [srv.submit(dA, dB, sync=False) for dA, dB in dev]
        states = drain(srv, len(ids))
        sat = srv.stats()
    rejected = sum(1 for s_ in states.values() if s_ != "done")
    ms_srv = sat["elapsed_s"] * 1e3
    # plain path one product at a time (each waited for before the next, as it serves requests)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prods_plain = 0
    for dA, dB in dev:
        C = sp.multiply(dA, dB)
        torch.cuda.synchronize()
        del C
    ms_plain = (time.perf_counter() - t0) * 1e3
    lam = 0.8 * R / (ms_plain * 1e-3)
    arrival = np.array([r.arrival_s for r in reqs]) / lam
    # plain path at rate lam: each request runs when it has arrived and the previous one is done
    lat_plain = []
    t0 = time.perf_counter()
    for k in range(R):
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
        drain(srv, R)
        th.join()
        live = srv.stats()
    gf = lambda p, ms: round(2.0 * p / (ms * 1e-3) / 1e9, 3)
    products = sat["products"]
    n_lap = sum(1 for r in reqs if r.kind == "lap3d")
    return {
        "workload": f"serve{R}", "value": gf(products, ms_srv), "unit": UNIT, "ms_per_step": round(ms_srv, 3),
        "steps": 1, "warmup": warmup, "requests": R, "products_per_step": products,
        "plain_value": gf(products, ms_plain), "plain_ms_per_step": round(ms_plain, 3),
        "speedup_vs_plain": round(ms_plain / ms_srv, 3), "rejected_over_cap": rejected,
        "server_jobs_per_s": round(sat["jobs_per_s"], 1), "mean_batch_jobs": round(sat["mean_batch_jobs"], 2),
        "splits": sat["splits"], "bytes_peak": sat["bytes_peak"], "gpu_launches": int(sat["kernel_launches"]),
        "latency": {"rate_per_s": round(lam, 2),
                    "what": "arrival to completion, ms, at 0.8 x the job rate of the plain path run one product "
                            "at a time",
                    "server_p50_ms": round(live["latency_p50_ms"], 3), "server_p99_ms": round(live["latency_p99_ms"], 3),
                    "server_max_ms": round(live["latency_max_ms"], 3),
                    "plain_p50_ms": round(_pct(lat_plain, 0.5), 3), "plain_p99_ms": round(_pct(lat_plain, 0.99), 3),
                    "plain_max_ms": round(max(lat_plain), 3),
                    "server_mean_batch_jobs": round(live["mean_batch_jobs"], 2),
                    "submit_lag_max_ms": round(lag[0] * 1e3, 3)},
        "description": f"{R} requests of a Poisson stream (seed 0): {R - n_lap} jobs A_j*B_j of the batch "
                       f"distribution drawn from its first {SERVE_POOL} jobs (request i takes job i mod "
                       f"{SERVE_POOL}), {n_lap} A*A for 3D 7-point Laplacians with g in 64..128 (one per g); "
                       f"FP64; 32 GB admission cap; inputs resident on the device; warm-up: {warmup} x (16 "
                       f"plain products + 200 served requests)",
    }


def _pinned(n: int, dtype, torch, registered: list):
    """Page-locked host array of exactly n elements (numpy memory registered with CUDA); the
    registered pointers are appended to `registered`, to be unregistered before the memory is
    freed (a stale registration over reused host memory breaks later copies)."""
    import mmap
    nbytes = max(n, 1) * np.dtype(dtype).itemsize
    try:
        # anonymous memory advised for transparent huge pages: after other work has fragmented
        # the host's memory, 4 KB pages slowed the copy of C to the host several times over
        buf = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        if hasattr(mmap, "MADV_HUGEPAGE"):
            buf.madvise(mmap.MADV_HUGEPAGE)
        a = np.frombuffer(buf, dtype=dtype, count=max(n, 1))
    except (OSError, ValueError, AttributeError):
        a = np.empty(max(n, 1), dtype=dtype)
    t = torch.from_numpy(a)
    rc = torch.cuda.cudart().cudaHostRegister(t.data_ptr(), t.numel() * t.element_size(), 0)
    if int(rc) == 0:
        registered.append(t.data_ptr())
    return t, (int(rc) == 0)


def run_e2e(args, mats, nnz_c, products_step, sp, torch, dist):
    """Same metric through spgemm_multiply_host: host A -> device, product, C -> host.
    Host arrays are page-locked; the output arrays are sized from nnz(C) of the device run."""
    hosts = []
    pinned_ok = True
    registered = []
    for name, M in mats:
        rp, ok1 = _pinned(M.rows + 1, np.int32, torch, registered)
        col, ok2 = _pinned(M.nnz, np.int32, torch, registered)
        val, ok3 = _pinned(M.nnz, np.float64, torch, registered)
        rp.copy_(torch.from_numpy(M.row_ptr.astype(np.int32)))
        col[:M.nnz].copy_(torch.from_numpy(M.col))
        val[:M.nnz].copy_(torch.from_numpy(M.val))
        hA = sp.DeviceCSR(M.rows, M.cols, rp, col[:M.nnz], val[:M.nnz])
        nnz = nnz_c[name]
        idx64 = nnz >= 2**31
        orp, o1 = _pinned(M.rows + 1, np.int64 if idx64 else np.int32, torch, registered)
        ocol, o2 = _pinned(nnz, np.int32, torch, registered)
        oval, o3 = _pinned(nnz, np.float64, torch, registered)
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
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    ws, _, _ = _dist()
    t = _max_over_ranks(float(np.mean(times)), dist, "cuda")
    torch.cuda.synchronize()
    h2d, d2h = int(sum(h[4] for h in hosts)), int(sum(h[5] for h in hosts))
    hosts.clear()
    for ptr in registered:
        torch.cuda.cudart().cudaHostUnregister(ptr)
    return {"value": round(_job_gflops(products_step, ws, t * 1e3), 3), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": round(t * 1e3, 3), "steps": e2e_steps,
            "host_buffers": "pinned" if pinned_ok else "pageable (pinning failed)",
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


def cpu_baseline_error(mats, res, seconds: float, sp) -> tuple:
    """CPU-baseline leg of an FP32 workload: the oracle on a seeded row sample (every row with at
    least 2^22 partial products plus random rows, about `seconds` of work), timed and
    extrapolated to the workload by products; and the max relative entry error of the GPU
    product `res` on those rows against the FP64 oracle."""
    import oracle
    total_t = total_p = 0.0
    worst = 0.0
    samples = []
    threads = 0
    for (name, M), (_, plan, C) in zip(mats, res):
        P = oracle.products_per_row(M, M)
        heavy = np.nonzero(P >= (1 << 22))[0]
        rng = np.random.default_rng(4321)
        budget = max(int(seconds * 2e8) - int(P[heavy].sum()), 0)
        order = rng.permutation(M.rows)
        k = int(np.searchsorted(np.cumsum(P[order]), budget)) + 1
        rows = np.unique(np.concatenate([heavy, order[:k]])).astype(np.int64)
        t = time.perf_counter()
        ref = oracle.spgemm(M, M, rows=rows)
        dt = time.perf_counter() - t
        threads = max(threads, ref.threads)
        sampled = int(P[rows].sum())
        total_t += int(P.sum()) * dt / max(sampled, 1)
        total_p += int(P.sum())
        rp = C.row_ptr.cpu().numpy().astype(np.int64)
        for t_, i in enumerate(rows):
            s_, e_ = int(rp[i]), int(rp[i + 1])
            r = slice(ref.row_ptr[t_], ref.row_ptr[t_ + 1])
            if e_ == s_:
                continue
            v = C.val[s_:e_].cpu().numpy().astype(np.float64)
            nz = np.abs(ref.val[r]) > 0
            if nz.any():
                worst = max(worst, float((np.abs(v - ref.val[r])[nz] / np.abs(ref.val[r][nz])).max()))
        samples.append(f"{name}: {len(rows)} rows ({len(heavy)} with >= 2^22 products), {sampled} products "
                       f"in {dt:.2f} s")
    cpu = {"value": round(2.0 * total_p / total_t / 1e9, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": "; ".join(samples) + " (time extrapolated to the whole workload by products)"}
    return cpu, worst


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
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--config", default=None, choices=["uniform10k", "plan_reuse", "rmat20_f32c", "batch4096", "serve20000"],
                    help="run one of the other configurations alone")
    ap.add_argument("--no-configs", action="store_true",
                    help="headline workload only (skip the uniform, FP32, batching and serving configs)")
    ap.add_argument("--side-steps", type=int, default=3, help="timed steps of the FP32 config")
    ap.add_argument("--side-warmup", type=int, default=3, help="warm-up steps of the other configs (>= 3)")
    ap.add_argument("--e2e-steps", type=int, default=5, help="timed steps of the end-to-end leg (<= --steps)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-accumulate", type=int, default=0, choices=[0, 1, 2],
                    help="FP64 sums: 0 shared atomics (default), 1 exact fixed point on the windowed rows, "
                         "2 deterministic (every row windowed, exact)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-products-per-step", type=float, default=2e8)
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--serve-requests", type=int, default=SERVE_REQUESTS)
    ap.add_argument("--serve-window-us", type=int, default=300)
    ap.add_argument("--serve-streams", type=int, default=2)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        sys.stderr.write("note: fewer than 3 warm-up steps\n")
    if args.impl == "reference":
        line, rank = run_reference(args)
    elif args.config:
        line, rank = run_one_config(args)
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
