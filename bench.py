#!/usr/bin/env python3
"""Throughput of the IFDLBM step on GB300 (MLUPS), one JSON line on rank 0.

Default workload: the batched parameter sweep of 64 cavities (grids drawn
from {129^2, 257^2, 385^2, 513^2}, theta from {30, 45, 60, 75, 90} deg,
n ~ U[0.5, 1.5], Re from {100, 400, 1000}; 566 MB of state, more than L2)
advanced together, one batched time step per bench step (Steps (2)-(8) of
the paper: equilibrium, lagged power-law relaxation time, the two-stage
finite-difference update on the mapped grid, wall nodes and the Eq. (2.19)
residual). Every timed step is bracketed by CUDA events on the library's
stream; a 256 MiB buffer is written between steps (outside the events) so
that no step starts from a warm L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32dev|fp64]
                  [--workload batch64|sweep257|...] [--impl ours|reference]

With N > 1 (torchrun), every rank advances its own copy of the workload
(independent cavities, no collective on the data path: weak scaling) and
the value is all ranks' lattice updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import atexit
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HEADLINE_METRIC = "MLUPS & HBM GB/s vs ~8 TB/s peak; FP32/batched vs FP64 at stated error"
KERNEL_NAMES = {0: "collide", 1: "half", 2: "full", 3: "reduce", 4: "fused"}
DEVICE_KERNEL = {"collide": "k_collide", "half": "k_half", "full": "k_full",
                 "reduce": "k_residual_reduce", "fused": "k_fused"}
# Algorithmic DRAM bytes per lattice update of each step kernel: every array
# element the kernel must read or write, once.
# The relaxation-time plane is stored in the storage type (FP32 in the
# FP32-deviation form: 9 x 4 x 2 + 4 + 4 = 80 B for the fused step).
ALGO_BYTES = {
    ("fused", "fp32dev"): 80, ("fused", "fp64"): 160,
    ("collide", "fp32dev"): 140, ("collide", "fp64"): 256,
    ("half", "fp32dev"): 76, ("half", "fp64"): 152,
    ("full", "fp32dev"): 132, ("full", "fp64"): 240,
}
# General quadrilaterals: the staged stencil kernels also read the per-node
# FP64 metrics (xi_x, xi_y, eta_x, eta_y; k_full also J); the fused FP32 kernel
# their FP32 roundings (c xi_x, c xi_y, c eta_x, c eta_y, J).
ALGO_BYTES_GENERAL = {"half": 32, "full": 40, "fused": 20}
FALLBACK_HBM_GBS = 6800.0
# GB300 instruction issue: 152 SMs x 4 schedulers, one warp instruction per clock each,
# at the maximum SM clock (MHz)
ISSUE_SLOTS_PER_CLOCK = 152 * 4
SM_MAX_MHZ = 2070.0


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--workload", default="batch64")
    p.add_argument("--precision", default="fp32dev", choices=["fp32dev", "fp64"])
    p.add_argument("--kernel", default="auto", choices=["auto", "staged", "fused"])
    p.add_argument("--lambda-mode", default="lagged", choices=["lagged", "implicit"],
                   help="relaxation time of Eq. (2.14): lagged (the paper's) or implicit")
    p.add_argument("--power-fp32", action="store_true",
                   help="fp32dev opt-in: power law of Eq. (1.4) in FP32 (outside the FP32 "
                        "deviation form, which keeps it in FP64)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-adjoint", action="store_true",
                   help="skip the adjoint measurement (257^2, 2000 steps, checkpoints every 100)")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="CPU work budget of the oracle baseline sample")
    p.add_argument("--fused-threads", type=int, default=0,
                   help="fix the fused kernel's CTA width (64/128/256) and skip the autotuner")
    p.add_argument("--fused-rows", type=int, default=0, help="rows per task with --fused-threads")
    p.add_argument("--schedule", default="grid", choices=["grid", "static", "dynamic"],
                   help="schedule with --fused-threads")
    return p.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# Clocks during the timed region (nvidia-smi sampler)
# ---------------------------------------------------------------------------
CLOCK_FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        self.marks = []

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            # ended on every exit path, an exception included: a sampler left
            # running would outlive the bench (and keep a profiler that waits
            # for the whole process tree waiting)
            atexit.register(self._reap)
        except Exception:
            self.proc = None

    def _reap(self):
        if self.proc is not None and self.proc.poll() is None:
            self.proc.kill()
            self.proc.wait()

    def mark(self):
        self.marks.append(time.time())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 10:
                        rows.append(parts)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = []
        reasons = set()
        sm_max = None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                clk = float(r[2])
                sm_max = float(r[3])
            except ValueError:
                continue
            if clk > 0:
                sm.append(clk)
            for k, name in enumerate(names):
                if r[6 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": sm_max, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# ncu-derived DRAM traffic (profiles/traffic.json), valid only for the
# kernel source it was taken from
# ---------------------------------------------------------------------------
KERNEL_SOURCES = {
    "fused": ["fused.cu", "d2q9.cuh", "fastpow.cuh", "reduce.cuh", "internal.h", "tma.cuh"],
    "collide": ["staged.cu", "d2q9.cuh", "fastpow.cuh", "reduce.cuh", "internal.h"],
    "half": ["staged.cu", "d2q9.cuh", "fastpow.cuh", "reduce.cuh", "internal.h"],
    "full": ["staged.cu", "d2q9.cuh", "fastpow.cuh", "reduce.cuh", "internal.h"],
}


def _code_only(text):
    """C/C++ source without comments and with whitespace runs collapsed, so that
    a comment edit does not retire the ncu record of unchanged code."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_digest(kernel="fused"):
    """Digest of the device code (comments and layout aside) a kernel is compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_07603_gb300", "csrc")
    for name in KERNEL_SOURCES.get(kernel, sorted(os.listdir(csrc))):
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode() + b"\0" + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _record(d, kernel, precision, workload):
    """The workload's own record, else (trapezoid workloads only) the kernel's."""
    e = d.get(f"{kernel}:{precision}:{workload}")
    if e is None and not is_general(workload):
        e = d[f"{kernel}:{precision}"]
    return e


def is_general(workload):
    """Workloads of general quadrilaterals (per-node metrics)."""
    return workload is not None and workload.startswith("quad")


def profile_record(kernel, precision, workload=None):
    """The ncu record of this kernel (and workload) if its sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = _record(d, kernel, precision, workload)
        return e if e.get("src_digest") == kernel_source_digest(kernel) else None
    except Exception:
        return None


def traffic_per_launch(kernel, precision, lu_per_launch, workload=None):
    """DRAM bytes per launch from the ncu record of this kernel (and workload,
    where one was captured: an L2-resident workload moves fewer bytes)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = _record(d, kernel, precision, workload)
        if e.get("src_digest") != kernel_source_digest(kernel):
            return None
        return float(e["bytes_per_lu"]) * lu_per_launch
    except Exception:
        return None


# ---------------------------------------------------------------------------
# Oracle CPU baseline (the only use of oracle/ in this file)
# ---------------------------------------------------------------------------
def oracle_run_of(O, spec):
    """The oracle's rest-state run of one workload cavity (trapezoid or quadrilateral)."""
    if hasattr(spec, "corners"):
        return O.quad_run(spec.nx, spec.ny, spec.corners, spec.Re, spec.n, H=spec.H, U=spec.U_lid)
    return O.cavity_run(spec.nx, spec.Re, spec.n, theta_deg=spec.theta_deg, U=spec.U_lid,
                        L=spec.L, H=spec.H, ny=spec.ny)


def spec_label(spec):
    shape = "quadrilateral" if hasattr(spec, "corners") else f"theta={spec.theta_deg:g}"
    return f"{shape}, n={spec.n:g}, Re={spec.Re:g}"


def oracle_sample_mlups(spec, seconds):
    """Times the FP64 oracle on one cavity of the workload from rest for about
    `seconds` of single-threaded NumPy work. Returns (MLUPS, steps, seconds)."""
    import oracle as O

    run = oracle_run_of(O, spec)
    t0 = time.perf_counter()
    run.advance(2)
    per = (time.perf_counter() - t0) / 2
    n = max(1, int(seconds / max(per, 1e-6)) - 2)
    t0 = time.perf_counter()
    run.advance(n)
    dt = time.perf_counter() - t0
    return spec.nodes * n / dt / 1e6, n, dt, run


def _oracle_worker(specs, warmup, steps, barrier, queue):
    """One process of the oracle pool: its cavities from rest, `warmup` steps,
    then (after every process is ready) `steps` steps of each, timed."""
    import oracle as O

    runs = [oracle_run_of(O, sp) for sp in specs]
    for r in runs:
        r.advance(warmup)
    barrier.wait(timeout=900)
    t0 = time.perf_counter()
    for _ in range(steps):
        for r in runs:
            r.advance(1)
    queue.put((sum(sp.nodes for sp in specs) * steps, time.perf_counter() - t0))


def oracle_pool_mlups(specs, warmup, steps, workers):
    """The oracle as it stands, one single-threaded process per group of
    cavities (spawned: the caller may hold a CUDA context), all started
    together: (whole-job MLUPS, wall seconds, processes)."""
    import multiprocessing

    workers = max(1, min(workers, len(specs)))
    ctx = multiprocessing.get_context("spawn")
    barrier = ctx.Barrier(workers + 1)
    queue = ctx.Queue()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                            "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    procs = [ctx.Process(target=_oracle_worker, args=(specs[k::workers], warmup, steps, barrier,
                                                      queue)) for k in range(workers)]
    try:
        for p in procs:
            p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    import queue as queue_mod
    import threading

    def fail(why):
        for p in procs:
            if p.is_alive():
                p.terminate()
        raise RuntimeError(f"oracle pool: {why}")

    try:
        barrier.wait(timeout=600)
    except threading.BrokenBarrierError:
        fail("a worker did not start (exit codes %s)" % [p.exitcode for p in procs])
    t0 = time.perf_counter()
    done = []
    while len(done) < workers:
        try:
            done.append(queue.get(timeout=5))
        except queue_mod.Empty:
            if any(p.exitcode not in (None, 0) for p in procs):
                fail("a worker failed (exit codes %s)" % [p.exitcode for p in procs])
    wall = time.perf_counter() - t0
    for p in procs:
        p.join(timeout=60)
    return sum(d[0] for d in done) / wall / 1e6, wall, workers


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(specs, seconds):
    """The oracle on the host cores: a single-thread sample of one cavity, and
    every cavity of the workload at once, one process per cavity (as many as
    there are cores), each for about `seconds`."""
    spec = specs[min(1, len(specs) - 1)]
    mlups, n, dt, _ = oracle_sample_mlups(spec, seconds)
    cores = host_cores()
    workers = min(cores, len(specs))
    # steps for about `seconds` of the largest process group at the sampled rate
    group_nodes = max(sum(sp.nodes for sp in specs[k::workers]) for k in range(workers))
    steps = max(2, int(seconds * mlups * 1e6 / group_nodes))
    pool, wall, used = oracle_pool_mlups(specs, 1, steps, workers)
    return {"value": round(pool, 4), "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": f"FP64 NumPy oracle, all {len(specs)} cavities of the workload from rest, "
                      f"{steps} steps each, one single-threaded process per cavity group on "
                      f"{used} of {cores} host cores, {wall:.1f} s",
            "single_core": {"value": round(mlups, 4), "cores": 1,
                            "sample": f"one {spec.nx}x{spec.ny} cavity ({spec_label(spec)}) from "
                                      f"rest, {n} steps in {dt:.1f} s, single thread"}}


# ---------------------------------------------------------------------------
# The GPU arm
# ---------------------------------------------------------------------------
LAMBDA_MODE = "lagged"  # set from --lambda-mode
POWER_FP32 = False      # set from --power-fp32


def make_solver(specs, precision, kernel, stream=None, workload=None, **extra):
    from paper_2306_07603_gb300.solver import Solver, cavity
    from paper_2306_07603_gb300.workloads import WORKLOAD_OPTIONS

    from paper_2306_07603_gb300.solver import quad_cavity
    cavs = [quad_cavity(s.nx, s.ny, s.corners, s.Re, s.n, U_lid=s.U_lid, H=s.H)
            if hasattr(s, "corners") else
            cavity(s.nx, s.ny, s.Re, s.n, theta_deg=s.theta_deg, U_lid=s.U_lid, L=s.L, H=s.H)
            for s in specs]
    opts = dict(WORKLOAD_OPTIONS.get(workload, {}), **extra)
    if LAMBDA_MODE != "lagged":
        opts["lambda_mode"] = LAMBDA_MODE
    if POWER_FP32:
        opts["power_fp32"] = True
    return Solver(cavs, stream=stream, precision=precision, kernel=kernel, **opts)


def tuning_options(tuning):
    names = {0: "grid", 1: "static", 2: "dynamic"}
    return dict(fused_threads=tuning.fused_threads, fused_rows=tuning.fused_rows,
                schedule=names[tuning.schedule])


def one_by_one_mlups(specs, precision, kernel, workload, steps, layout):
    """The same cavities as separate handles, stepped one after another each
    time step (one launch per cavity instead of one per batch)."""
    import torch

    from paper_2306_07603_gb300 import capi

    stream = torch.cuda.Stream()
    solvers = [make_solver([sp], precision, kernel, stream=stream, workload=workload, **layout)
               for sp in specs]
    for s in solvers:
        s.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        for s in solvers:
            capi.ifdlbm_step(s.h, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    for s in solvers:
        s.close()
    return sum(sp.nodes for sp in specs) * steps / (ms * 1e-3) / 1e6


def reduce_over_ranks(total_ms, launches, world, device):
    """Slowest rank's timed milliseconds and the job's total kernel launches."""
    import torch
    import torch.distributed as dist

    t_ms = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    t_n = torch.tensor([float(launches)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
        dist.all_reduce(t_n, op=dist.ReduceOp.SUM)
    return float(t_ms[0]), int(t_n[0])


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.workloads import WORKLOADS

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    specs = WORKLOADS[args.workload]()
    lu_step = sum(s.nodes for s in specs)

    fixed = {}
    if args.fused_threads:
        fixed = dict(fused_threads=args.fused_threads, fused_rows=args.fused_rows,
                     schedule=args.schedule)
    s = make_solver(specs, args.precision, args.kernel, workload=args.workload, **fixed)
    stream = s.stream
    tuning = None
    if capi.ifdlbm_info(s.h, 0).fused_threads and not fixed:
        tuning = s.autotune(trial_steps=10)           # layout and schedule, state unchanged
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sampler = ClockSampler(local)
    sampler.start()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(0.0)
            s.step(1)
    s.sync()
    capi.ifdlbm_profile(s.h, 1)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = capi.ifdlbm_launch_count()
    sampler.mark()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            capi.ifdlbm_step(s.h, 1)
            ends[k].record(stream)
    torch.cuda.synchronize()
    sampler.mark()
    launches = capi.ifdlbm_launch_count() - launches0
    if world > 1:
        dist.barrier()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    kern = {}
    for kid, name in KERNEL_NAMES.items():
        ms, n = capi.ifdlbm_profile_read(s.h, kid)
        if n:
            kern[name] = (ms, n)
    capi.ifdlbm_profile(s.h, 0)
    resid = s.residual()
    clocks = sampler.stop()

    max_ms, launches_all = reduce_over_ranks(total_ms, launches, world, "cuda")
    value = lu_step * world * args.steps / (max_ms * 1e-3) / 1e6

    general = is_general(args.workload)
    # roofline of the dominant kernel, from its live event times
    peak, peak_src = load_peaks()
    dom = max(kern, key=lambda k: kern[k][0]) if kern else None
    roofline = None
    if dom is not None and (dom, args.precision) in ALGO_BYTES:
        ms, n = kern[dom]
        per_launch_s = ms / n * 1e-3
        algo = (ALGO_BYTES[(dom, args.precision)] +
                (ALGO_BYTES_GENERAL.get(dom, 0) if general else 0)) * lu_step
        achieved = algo / per_launch_s / 1e9
        roofline = {"bound": "hbm", "kernel": DEVICE_KERNEL[dom], "achieved": round(achieved, 1),
                    "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "traffic": traffic_per_launch(dom, args.precision, lu_step, args.workload)
                    if args.lambda_mode == "lagged" and not args.power_fp32 else None,
                    "algorithmic_bytes": algo, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"
                    if peak_src == "measured" else "fallback",
                    "time_share": round(ms / sum(v[0] for v in kern.values()), 4)}

    # what bounds the step before HBM does, from the ncu record of the same
    # kernel sources: the FP64 pipe (1/64 of the FP32 rate on GB300; the FP64
    # form) and the schedulers' instruction issue (the FP32-deviation form)
    # (the ncu records are of the lagged kernels)
    rec = (profile_record(dom, args.precision, args.workload)
           if dom is not None and args.lambda_mode == "lagged" and not args.power_fp32 else None)
    fp64 = issue = None
    if rec is not None and "fp64_pipe_pct_elapsed" in rec:
        fp64 = {"bound": "alu", "unit": "fraction of the FP64 pipe's peak issue rate",
                "frac": round(rec["fp64_pipe_pct_elapsed"] / 100.0, 3),
                "source": rec["source"] + " (ncu sm__inst_executed_pipe_fp64, elapsed)"}
    if rec is not None and "issue_active_pct" in rec:
        issue = {"bound": "issue", "unit": "fraction of cycles the SM schedulers issue",
                 "frac": round(rec["issue_active_pct"] / 100.0, 3),
                 "source": rec["source"] + " (ncu smsp__issue_active, active cycles)"}
        if "warp_inst_per_node" in rec and dom is not None:
            # the same bound from this run's own timing: warp instructions per node (ncu,
            # same kernel sources) x nodes per launch / launch time, against the issue
            # peak of 152 SMs x 4 schedulers x 1 instruction per clock at the max clock
            ms, n = kern[dom]
            rate = rec["warp_inst_per_node"] * lu_step / (ms / n * 1e-3) / 1e9
            peak_issue = ISSUE_SLOTS_PER_CLOCK * SM_MAX_MHZ * 1e6 / 1e9
            issue.update({"achieved": round(rate, 1), "peak": round(peak_issue, 1),
                          "unit": "G warp instructions/s",
                          "frac": round(rate / peak_issue, 4),
                          "issue_active_ncu": round(rec["issue_active_pct"] / 100.0, 3),
                          "warp_inst_per_node": rec["warp_inst_per_node"]})
    layout = fixed or (tuning_options(tuning) if tuning is not None else {})
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, specs, stream, world, layout)
    batch = None
    if len(specs) > 1 and rank == 0:
        batch = {"cavities": len(specs), "batched_mlups": None,
                 "one_by_one_mlups": round(one_by_one_mlups(specs, args.precision, args.kernel,
                                                            args.workload, max(5, args.steps // 4),
                                                            layout), 2)}

    out = None
    if rank == 0:
        step_ms = max_ms / args.steps
        out = {
            "metric": "MLUPS",
            "value": round(value, 2),
            "unit": "MLUPS",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(step_ms, 5),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "fp32dev" else "f64",
            "data": "synthetic (cavities from rest; no dataset)",
            "config": {"workload": args.workload, "cavities": len(specs),
                       "grids": sorted({f"{sp.nx}x{sp.ny}" for sp in specs}),
                       "lattice_updates_per_step": lu_step, "precision": args.precision,
                       "kernel": args.kernel, "lambda_mode": args.lambda_mode,
                       "power_law": "fp32 (opt-in)" if args.power_fp32 else "fp64",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": "256 MiB buffer written between timed steps (outside the events)",
                       "metric_definition": HEADLINE_METRIC},
            "hbm_gbs_algorithmic": round(value * 1e6 * (80 if args.precision == "fp32dev" else 160) / 1e9, 1),
            "roofline": roofline,
            "roofline_fp64": fp64,
            "roofline_issue": issue,
            "kernels_ms_per_launch": {k: round(v[0] / v[1], 5) for k, v in kern.items()},
            "gpu_launches": launches_all,
            "clocks": clocks,
            "e2e": e2e,
            "last_residual_cavity0": [float(x) for x in resid[0]],
        }
        if fixed:
            out["config"]["fused_layout"] = fixed
        if tuning is not None:
            out["config"]["autotuned"] = {"fused_threads": tuning.fused_threads,
                                          "fused_rows": tuning.fused_rows,
                                          "schedule": ["grid", "static", "dynamic"][tuning.schedule],
                                          "tasks": tuning.ntasks, "candidates": tuning.candidates}
        if batch is not None:
            batch["batched_mlups"] = out["value"]
            out["batch"] = batch
        if world == 1 and not args.no_adjoint:
            out["adjoint"] = run_adjoint_measure()
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(specs, args.cpu_seconds)
    s.close()
    if world > 1:
        dist.destroy_process_group()
    return out


def run_adjoint_measure(nx=257, ny=257, T=2000, every=100, n=0.75, Re=400.0, theta=60.0):
    """Time and memory of d E(T) / d(n, Re, theta) through the hand-written
    adjoint against the plain FP64 forward run of the same T steps."""
    import torch

    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.adjoint import KineticEnergy
    from paper_2306_07603_gb300.solver import Solver, cavity

    s = Solver([cavity(nx, ny, Re, n, theta_deg=theta)], precision="fp64", kernel="staged",
               dt_mode="grid")   # the time-step rule the adjoint uses (dt independent of theta)
    s.step(2)
    s.sync()
    t0 = time.perf_counter()
    s.step(T)
    s.sync()
    t_plain = time.perf_counter() - t0
    state_bytes = capi.ifdlbm_state_bytes(s.h)
    inter_bytes = capi.ifdlbm_intermediate_bytes(s.h)
    handle_bytes = capi.ifdlbm_info(s.h, 0).device_bytes
    s.close()
    def timed(ev):
        p = torch.tensor([n, Re, theta], dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = KineticEnergy.apply(p, nx, ny, T, ev)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        J.backward()
        torch.cuda.synchronize()
        return p, J, t_fwd, time.perf_counter() - t0

    p, J, t_fwd, t_bwd = timed(every)
    # no recomputation: the forward pass keeps every state and its intermediates
    p1, _, t_fwd1, t_bwd1 = timed(1)
    torch.cuda.empty_cache()
    ckpt = (T + every - 1) // every + 1
    return {"workload": f"{nx}x{ny}, theta={theta:g}, n={n:g}, Re={Re:g}, {T} steps, FP64, "
                        f"checkpoint every {every}",
            "plain_forward_s": round(t_plain, 4), "forward_with_checkpoints_s": round(t_fwd, 4),
            "backward_s": round(t_bwd, 4), "gradient_over_forward": round((t_fwd + t_bwd) / t_plain, 2),
            "checkpoint_bytes": ckpt * state_bytes,
            "segment_bytes": every * (state_bytes + inter_bytes),   # states + intermediates
            "handle_bytes": handle_bytes, "adjoint_scratch_bytes": 4 * 9 * state_bytes // 10,
            "dJ": {"n": float(p.grad[0]), "Re": float(p.grad[1]), "theta_deg": float(p.grad[2])},
            "J": float(J.detach()),
            "keep_all": {"forward_s": round(t_fwd1, 4), "backward_s": round(t_bwd1, 4),
                         "gradient_over_forward": round((t_fwd1 + t_bwd1) / t_plain, 2),
                         "bytes": (T + 1) * state_bytes + T * inter_bytes,
                         "same_gradient": bool(torch.equal(p1.grad, p.grad))}}


def run_e2e(args, specs, stream, world, layout=None):
    """Same metric through the public API with HOST buffers: create the batch
    from host parameters, then every step's residuals and divergence word come
    back into pinned host memory and are read by the host (step n's while step
    n + 1 runs: ifdlbm_batch_residual_async, an event per step), and the final
    fields of every cavity come back to the host. The window covers all of it,
    over at least 200 steps; the creation time (parameters and metrics to the
    device, allocation) is also reported on its own, with the rate of the
    stepping part alone."""
    import numpy as np
    import torch

    from paper_2306_07603_gb300 import capi

    nsteps = max(200, args.steps)
    ncav = len(specs)
    res = [torch.empty((ncav, 4), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    st = [torch.zeros(1, dtype=torch.int32, pin_memory=True) for _ in range(2)]
    ev = [torch.cuda.Event() for _ in range(2)]
    hist = np.empty((nsteps, ncav, 4))
    fields = [torch.empty((4, sp.ny, sp.nx), dtype=torch.float64, pin_memory=True) for sp in specs]

    def take(n):  # the host reads step n's residuals
        ev[n % 2].synchronize()
        if int(st[n % 2][0]) & 1:
            raise RuntimeError(f"step {n} produced a non-finite velocity")
        hist[n] = res[n % 2].numpy()

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = make_solver(specs, args.precision, args.kernel, stream=stream, workload=args.workload,
                    **(layout or {}))
    t_created = time.perf_counter()
    for n in range(nsteps):
        capi.ifdlbm_step(s.h, 1)
        capi.ifdlbm_batch_residual_async(s.h, res[n % 2], st[n % 2])
        ev[n % 2].record(s.stream)
        if n > 0:
            take(n - 1)
    take(nsteps - 1)
    for k in range(ncav):
        f = fields[k].numpy()
        capi.ifdlbm_batch_macros(s.h, k, f[0], f[1], f[2], f[3])
    t1 = time.perf_counter()
    h2d = capi.ifdlbm_info(s.h, 0).h2d_bytes
    s.close()
    if not np.all(np.isfinite(hist)):
        raise RuntimeError("non-finite residual in the end-to-end run")
    lu = sum(sp.nodes for sp in specs) * nsteps * world
    d2h = (ncav * 4 * 8 + 4) * nsteps + sum(4 * 8 * sp.nodes for sp in specs)
    return {"value": round(lu / (t1 - t0) / 1e6, 2), "unit": "MLUPS",
            "h2d_bytes_per_step": round(h2d / nsteps, 1), "d2h_bytes_per_step": round(d2h / nsteps, 1),
            "steps": nsteps, "create_s": round(t_created - t0, 4),
            "stepping_mlups": round(lu / (t1 - t_created) / 1e6, 2),
            "what": "create from host parameters + every step's residuals and divergence word "
                    "D2H into pinned memory, read by the host one step behind the device "
                    "(ifdlbm_batch_residual_async + event) + final rho/u/v/psi D2H"}


# ---------------------------------------------------------------------------
# The reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    from paper_2306_07603_gb300.workloads import WORKLOADS

    rank, world, _ = dist_env()
    if rank != 0:
        return None
    specs = WORKLOADS[args.workload]()
    # one reference step = one time step of every cavity of the workload, the
    # cavities spread over one single-threaded oracle process per host core
    cores = host_cores()
    value, dt, used = oracle_pool_mlups(specs, args.warmup, args.steps, cores)
    return {
        "impl": "reference", "metric": "MLUPS", "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "precision": "fp64 oracle",
                   "sample": "each step = one time step of every cavity of the workload"},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": used, "kind": "oracle",
                         "sample": f"{args.steps} steps of all {len(specs)} cavities from rest, "
                                   f"one single-threaded NumPy process per cavity group on "
                                   f"{used} of {cores} host cores"},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    global LAMBDA_MODE, POWER_FP32
    args = parse_args(argv)
    LAMBDA_MODE = args.lambda_mode
    POWER_FP32 = args.power_fp32
    if args.power_fp32 and args.precision != "fp32dev":
        raise SystemExit("--power-fp32 needs --precision fp32dev")
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
