#!/usr/bin/env python
"""Benchmark of the OECDG forward step (arXiv:2503.12473) on GB300.

Workload: 2D Euler (gamma = 1.4) OECDG, Q^2 tensor Legendre basis, 1024 x 1024
primal mesh + dual mesh shifted by (h/2, h/2), [0,1]^2 transmissive, SSP-RK3,
CFL 0.1, four-quadrant Riemann data split at (0.8, 0.8) (synthetic, seeded-free
closed-form data).  A "step" is one SSP-RK3 time step: the wave-speed
reduction, then three stages of (CDG right-hand side + RK combine, sigma
reduction, OE damping).

Metric: FP64 DOF-updates per second per RK stage = 3 * DOF * steps / time,
DOF = 2 meshes x 4 fields x 9 modes x 1024^2 = 75,497,472.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per rank, launched by torchrun); the
value is the sum over ranks of the work divided by the max over ranks of the
time.  The reference arm times the CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FP64 DOF-updates/s per RK stage, 2D Euler 1024^2 k=2"
UNIT = "DOF-updates/s"

# Peaks (per GPU).  HBM: the measured copy bandwidth of the GB300s.
# FP64: 152 SMs x 2 FP64 FMA per SM per clock x 2 flops x 2.07 GHz (the nominal
# 1.25 TFLOP/s at the maximum SM clock); a DFMA-throughput probe measured 1.19
# TFLOP/s at 1.99 GHz, i.e. the same 2 FMA per SM per clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
HBM_FALLBACK_GBS = 6800.0

# Algorithmic FP64 flops per cell (one primal or dual cell, 2D Euler Q^2) of
# the two hot kernels, counted from the executed FP64 instructions of one
# launch (2 x DFMA + DADD + DMUL) divided by the cells of the launch: the
# kernels are fully unrolled, so this is the arithmetic of the algorithm as
# implemented.  The stage kernel's first stage (no u^n term) does 6,899 per
# cell, the other two 6,971: the figure is their mean over a step.  Source: an
# ncu capture of the FP64 instruction counters of the three stage and three OE
# launches of one 512^2 step.
FLOPS_PER_CELL = {"stage": 6947, "oe": 5808}
# DRAM bytes per cell per launch (ncu dram__bytes_read + write, same capture,
# mean over the step's launches); None once a kernel changes after the capture.
TRAFFIC_PER_CELL = {"stage": 828, "oe": 501}
# Algorithmic HBM bytes per cell: stage reads u_in (36 doubles) and, in two of
# three stages, u^n (36), writes u_h (36); OE reads u_h (36), writes u_sigma (36)
# (neighbour re-reads, of both meshes, are L2 hits: the two meshes' blocks of a
# tile run side by side).
BYTES_PER_CELL = {"stage": (36 + 24 + 36) * 8, "oe": (36 + 36) * 8}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        sm_sorted = sorted(sm)
        med = sm_sorted[len(sm_sorted) // 2] if sm_sorted else None
        return {"sm_mhz": med, "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def init_dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max_ms(ms: float, ws: int, device) -> float:
    """Max over ranks of a duration (the slowest replica sets the job time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_value(dof: int, steps: int, ws: int, ms_max: float) -> float:
    """Whole-job DOF-updates per second per RK stage: every rank advances its own
    replica of `dof` degrees of freedom by `steps` three-stage steps."""
    return 3.0 * dof * steps * ws / (ms_max * 1e-3)


def config_dict(n, dof):
    return {"workload": f"euler_2d_riemann_q2_{n}", "model": None, "nx": n, "ny": n, "k": 2, "basis": "Q",
            "system": "euler", "bc": "transmissive", "rk": "ssp-rk3", "cfl": 0.1, "oe": True, "dof": dof,
            "l2": (f"inputs larger than L2 (state {dof * 8 / 1e6:.0f} MB > 129 MB L2)" if dof * 8 > 129e6 else
                   f"state {dof * 8 / 1e6:.0f} MB fits in L2: not a bench configuration"),
            "parallelism": "replicas"}


# ---------------------------------------------------------------- oracle ---

def oracle_rate(steps: int, warmup: int, budget_s: float = 90.0):
    """Time the CPU oracle on the same workload at a bounded mesh size.  Returns
    (DOF-updates/s, cores, sample text, seconds per step)."""
    from oracle import oracle as O
    from paper_2503_12473_gb300 import workloads as W
    cores = O.num_threads()

    def run(n, k):
        w = W.riemann_2d(n=n)
        p = O.Problem(dim=2, nx=n, ny=n, k=2, system=O.EULER, bc=O.TRANSMISSIVE, cfl=0.1)
        u = O.project_fn(p, w.u0)
        t0 = time.perf_counter()
        O.advance(p, u, 0.0, 0.0, k)
        return time.perf_counter() - t0, u.size

    dt, dof = run(16, 1)
    rate = 3 * dof / dt
    per_step = budget_s / max(steps + warmup, 1)
    n = int(math.sqrt(per_step * rate / (3 * 72)))
    n = max(8, min(128, (n // 8) * 8))
    if warmup:
        run(n, warmup)
    dt, dof = run(n, steps)
    rate = 3 * dof * steps / dt
    sample = (f"four-quadrant Riemann data on a {n}x{n} Q^2 mesh (same workload, smaller mesh: the oracle's cost "
              f"per DOF-update does not depend on the mesh size), {steps} SSP-RK3 steps after {warmup} warm-up")
    return rate, cores, sample, dt / steps


def run_reference(args, ws, rank):
    if rank != 0:
        return
    steps, warmup = args.steps, args.warmup
    rate, cores, sample, sps = oracle_rate(steps, warmup)
    dof = 2 * 4 * 9 * args.n * args.n
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws, "steps": steps,
            "warmup": warmup, "ms_per_step": sps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(args.n, dof),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours ---

def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    from paper_2503_12473_gb300 import oecdg as G
    from paper_2503_12473_gb300 import workloads as W

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    G.load()
    n = args.n
    w = W.riemann_2d(n=n)
    stream = torch.cuda.Stream()
    ctx = G.Context(G.desc_from_workload(w), stream=stream)
    dof = ctx.cdg_state_numel()
    with torch.cuda.stream(stream):
        u0 = ctx.project(w.u0)
        # warm-up on a copy
        uw = u0.clone()
        if args.warmup:
            ctx.cdg_step_async(uw, 0.0, 0.0, args.warmup)
        stream.synchronize()
        st = ctx.cdg_check_status()
        if st != G.CDG_OK:
            raise G.CdgError(st, "warm-up")
        del uw
        u = u0.clone()
        stream.synchronize()

        def barrier():
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()

        clocks = ClockSampler(local)
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        launches0 = ctx.cdg_launch_count()
        ctx.cdg_profile_begin(3 * args.steps + 8)
        barrier()
        ev0.record(stream)
        ctx.cdg_step_async(u, 0.0, 0.0, args.steps)
        ev1.record(stream)
        barrier()
        clocks_res = clocks.stop()
        prof = ctx.cdg_profile_end()
        launches = ctx.cdg_launch_count() - launches0
        ms = ev0.elapsed_time(ev1)
        st = ctx.cdg_check_status()
        if st != G.CDG_OK:
            raise G.CdgError(st, "timed steps")
        t_final = ctx.cdg_get_time()
        ms_max = reduce_max_ms(ms, ws, "cuda")
        value = job_value(dof, args.steps, ws, ms_max)

        # end to end through the C-ABI with host buffers: each step copies the
        # state from pinned host memory, steps, and copies the result back
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        h_u = torch.empty(u0.shape, dtype=torch.float64, pin_memory=True)
        h_u.copy_(u0)
        d_u = torch.empty_like(u0)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            d_u.copy_(h_u, non_blocking=True)
            ctx.cdg_step_async(d_u, 0.0, 0.0, 1)
            h_u.copy_(d_u, non_blocking=True)
        e1.record(stream)
        barrier()
        e2e_ms = e0.elapsed_time(e1)
        e2e_value = job_value(dof, e2e_steps, ws, reduce_max_ms(e2e_ms, ws, "cuda"))
        state_bytes = dof * 8

    if ws > 1:
        dist.barrier()
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel, from the events of the timed region
    cells = 2 * n * n
    kname = "stage" if prof["stage"][0] >= prof["oe"][0] else "oe"
    kms, kcount = prof[kname]
    avg_s = (kms / max(kcount, 1)) * 1e-3
    fpc = FLOPS_PER_CELL[kname]
    peaks = measured_peaks()
    roof = {"bound": "alu", "kernel": f"k_{kname}2d (Euler, transmissive)", "unit": "TFLOP/s",
            "peak": FP64_PEAK_TFLOPS, "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz",
            "avg_launch_ms": avg_s * 1e3, "launches": kcount,
            "traffic": (TRAFFIC_PER_CELL[kname] * cells if TRAFFIC_PER_CELL[kname] is not None else None),
            "traffic_unit": "bytes per launch"}
    if fpc is not None:
        roof["achieved"] = fpc * cells / avg_s / 1e12
        roof["frac"] = roof["achieved"] / FP64_PEAK_TFLOPS
        roof["flops_per_cell"] = fpc
    else:
        roof["achieved"] = None
        roof["frac"] = None
    hbm_peak = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)
    roof["hbm"] = {"achieved_gbs": BYTES_PER_CELL[kname] * cells / avg_s / 1e9, "peak_gbs": hbm_peak,
                   "frac": BYTES_PER_CELL[kname] * cells / avg_s / 1e9 / hbm_peak,
                   "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    roof["kernel_share"] = {k: prof[k][0] / ms for k in ("stage", "oe")}
    # the other hot kernel, same arithmetic
    oname = "oe" if kname == "stage" else "stage"
    oms, ocount = prof[oname]
    if ocount and FLOPS_PER_CELL[oname] is not None:
        o_ach = FLOPS_PER_CELL[oname] * cells / ((oms / ocount) * 1e-3) / 1e12
        roof["other_kernel"] = {"kernel": f"k_{oname}2d", "avg_launch_ms": oms / ocount, "achieved": o_ach,
                                "frac": o_ach / FP64_PEAK_TFLOPS, "flops_per_cell": FLOPS_PER_CELL[oname]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(n, dof),
            "t_final": t_final, "roofline": roof,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes, "steps": e2e_steps},
            "gpu_launches": launches, "clocks": clocks_res}
    if ws == 1 and not args.no_cpu_baseline:
        rate, cores, sample, sps = oracle_rate(2, 0, budget_s=20.0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# Executed FP64 flops (2 DFMA + DADD + DMUL) and DRAM bytes per cell of the
# degree-generic 2D kernels, 2D Euler steady wave, periodic, 512^2; keys
# (k, basis).  Each figure is the mean over the launches of one step (the
# (k+1)-order RK method's 2, 3 or 4 stage and OE launches) of one ncu capture of
# the FP64 instruction counters and dram__bytes_read + write, divided by the
# 2 x 512^2 cells of a launch.  The P^1, P^2 and Q^1 states (50-101 MB) fit in
# L2, so their DRAM bytes fall below the algorithmic state traffic.
FLOPS_PER_CELL_2K = {
    (1, "P"): {"stage": 3309, "oe": 2511},
    (2, "P"): {"stage": 9523, "oe": 6785},
    (3, "P"): {"stage": 21711, "oe": 15164},
    (1, "Q"): {"stage": 3287, "oe": 2983},
    (3, "Q"): {"stage": 24694, "oe": 21492},
}
TRAFFIC_PER_CELL_2K = {
    (1, "P"): {"stage": 293, "oe": 196},
    (2, "P"): {"stage": 704, "oe": 614},
    (3, "P"): {"stage": 1593, "oe": 1271},
    (1, "Q"): {"stage": 374, "oe": 285},
    (3, "Q"): {"stage": 2191, "oe": 1509},
}


def run_generic(args, ws, rank, local):
    """2D Euler steady wave (the smooth test of Table 4): Q^k or P^k, k = 1..3,
    with the (k+1)-order RK method of the accuracy tests, on the degree-generic
    kernels; DOF-updates per second per RK stage and the roofline of the
    dominant kernel."""
    import torch
    from paper_2503_12473_gb300 import oecdg as G
    from paper_2503_12473_gb300 import workloads as W

    torch.cuda.set_device(local)
    G.load()
    k, basis = args.k, (W.BASIS_P if args.basis == "P" else W.BASIS_Q)
    n = args.n
    w = W.steady_wave_2d_workload(n, k, basis)
    stream = torch.cuda.Stream()
    ctx = G.Context(G.desc_from_workload(w), stream=stream)
    dof = ctx.cdg_state_numel()
    stages = 4 if w.rk == 4 else w.rk
    with torch.cuda.stream(stream):
        u = ctx.project(w.u0)
        ctx.cdg_step_async(u, 0.0, 0.0, args.warmup)
        stream.synchronize()
        if ctx.cdg_check_status() != G.CDG_OK:
            raise RuntimeError("warm-up reached a non-physical state")
        clocks = ClockSampler(local)
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        launches0 = ctx.cdg_launch_count()
        ctx.cdg_profile_begin(stages * args.steps + 8)
        torch.cuda.synchronize()
        ev0.record(stream)
        ctx.cdg_step_async(u, 0.0, 0.0, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks_res = clocks.stop()
        prof = ctx.cdg_profile_end()
        launches = ctx.cdg_launch_count() - launches0
        ms = ev0.elapsed_time(ev1)
        if ctx.cdg_check_status() != G.CDG_OK:
            raise RuntimeError("timed steps reached a non-physical state")
    if rank != 0:
        return
    cells = 2 * n * n
    kname = "stage" if prof["stage"][0] >= prof["oe"][0] else "oe"
    kms, kcount = prof[kname]
    avg_s = (kms / max(kcount, 1)) * 1e-3
    key = (k, args.basis)
    fpc = FLOPS_PER_CELL_2K.get(key, {}).get(kname)
    tpc = TRAFFIC_PER_CELL_2K.get(key, {}).get(kname)
    if k == 2 and args.basis == "Q" and w.rk != 4:
        fpc, tpc = FLOPS_PER_CELL[kname], None
    tiled = k == 2 and args.basis == "Q" and w.rk != 4  # served by the tiled Q^2 kernels
    roof = {"bound": "alu", "kernel": f"k_{kname}{'2d' if tiled else '2k'} (Euler, periodic, {args.basis}{k})",
            "unit": "TFLOP/s",
            "peak": FP64_PEAK_TFLOPS, "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz",
            "avg_launch_ms": avg_s * 1e3, "launches": kcount,
            "achieved": fpc * cells / avg_s / 1e12 if fpc else None,
            "frac": fpc * cells / avg_s / 1e12 / FP64_PEAK_TFLOPS if fpc else None,
            "flops_per_cell": fpc, "traffic": tpc * cells if tpc else None, "traffic_unit": "bytes per launch",
            "kernel_share": {q: prof[q][0] / ms for q in ("stage", "oe")}}
    line = {"metric": METRIC.replace("2D Euler 1024^2 k=2", f"2D Euler steady wave {n}^2 {args.basis}{k}"),
            "value": dof * stages * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "nx": n, "ny": n, "k": k, "basis": args.basis, "system": "euler",
                       "bc": "periodic", "rk": {2: "ssp-rk2", 3: "ssp-rk3", 4: "rk4"}[w.rk], "cfl": w.cfl,
                       "oe": True, "dof": dof,
                       "l2": (f"inputs larger than L2 (state {dof * 8 / 1e6:.0f} MB > 129 MB L2)"
                              if dof * 8 > 129e6 else f"state {dof * 8 / 1e6:.0f} MB fits in L2")},
            "roofline": roof, "gpu_launches": launches, "clocks": clocks_res}
    print(json.dumps(line), flush=True)


def run_time_to_solution(args, ws, rank, local):
    """The two 1D workloads run to their end time (1D advection, 128 cells,
    T = 2 pi; 1D Euler Shu-Osher, 4000 cells, T = 1.8): launch-bound, so the
    figure is the time to solution, with one launch per kernel
    (cdg_step_async), with the step replayed as a CUDA graph (cdg_step_graph)
    and with all steps in one persistent cooperative launch
    (cdg_step_persistent); the three results must be identical."""
    import torch
    from paper_2503_12473_gb300 import oecdg as G
    from paper_2503_12473_gb300 import workloads as W

    torch.cuda.set_device(local)
    G.load()
    w = W.advection_1d(128) if args.workload == "advection-1d" else W.shu_osher_1d(4000)
    stream = torch.cuda.Stream()
    ctx = G.Context(G.desc_from_workload(w), stream=stream)
    with torch.cuda.stream(stream):
        u0 = ctx.project(w.u0)
        # steps to T: one untimed pass, one step at a time
        uw = u0.clone()
        t, nsteps = 0.0, 0
        while t < w.T:
            ctx.cdg_step_async(uw, t, w.T, 1)
            t = ctx.cdg_get_time()
            nsteps += 1
        res = {}
        steppers = {"kernels": ctx.cdg_step_async, "graph": ctx.cdg_step_graph,
                    "persistent": ctx.cdg_step_persistent}
        for mode, step in steppers.items():
            u = u0.clone()
            step(u, 0.0, w.T, 3)  # warm-up (and, for the graph, its capture for this u)
            u.copy_(u0)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            l0 = ctx.cdg_launch_count()
            ev0.record(stream)
            step(u, 0.0, w.T, nsteps)
            ev1.record(stream)
            torch.cuda.synchronize()
            if ctx.cdg_check_status() != G.CDG_OK:
                raise RuntimeError("non-physical state")
            res[mode] = (ev0.elapsed_time(ev1), ctx.cdg_launch_count() - l0, u, ctx.cdg_get_time())
    same = bool(torch.equal(res["kernels"][2], res["graph"][2]) and torch.equal(res["kernels"][2], res["persistent"][2]))
    dof = ctx.cdg_state_numel()
    line = {"metric": f"time to solution, {w.name} to T = {w.T:.6g}", "workload": w.name, "steps": nsteps,
            "dof": dof, "t_final": res["persistent"][3],
            "identical": same, "unit_time": "ms", "higher_is_better": False, "dtype": "f64", "data": "synthetic"}
    for mode in steppers:
        line[mode] = {"ms": res[mode][0], "us_per_step": 1e3 * res[mode][0] / nsteps,
                      "gpu_launches": res[mode][1],
                      "dof_updates_per_s": 3.0 * dof * nsteps / (res[mode][0] * 1e-3)}
    line["speedup_graph"] = res["kernels"][0] / res["graph"][0]
    line["speedup_persistent"] = res["kernels"][0] / res["persistent"][0]
    print(json.dumps(line), flush=True)


def run_batched(args, ws, rank, local):
    """256 independent periodic 2D Euler Q^2 problems (seeded sizes in
    {64,...,512}^2 and data): all steps in one persistent cooperative launch
    (autotuned tile height and grid) against the graph-captured batched
    launches per phase and against per-instance launches of the same kernels,
    same steps; the three results must be identical."""
    import torch
    from paper_2503_12473_gb300 import oecdg as G
    from paper_2503_12473_gb300 import workloads as W

    torch.cuda.set_device(local)
    G.load()
    insts = W.batched_instances(seed=args.seed, count=args.count)
    descs = [G.MeshDesc(dim=2, nx=q.n, ny=q.n, system=G.EULER, bc=G.PERIODIC, cfl=0.1) for q in insts]
    stream = torch.cuda.Stream()
    ctxs = [G.Context(d, stream=stream) for d in descs]
    with torch.cuda.stream(stream):
        u0 = [c.project(W.batched_ic(q)) for c, q in zip(ctxs, insts)]
    stream.synchronize()
    dof = sum(u.numel() for u in u0)
    batch = G.Batch(descs, stream=stream)
    cache = os.path.join(ROOT, "paper_2503_12473_gb300", "_build", "batch_autotune.json")
    rows = batch.cdg_batch_autotune(u0, cache)
    ub = [u.clone() for u in u0]
    uw = [u.clone() for u in u0]
    batch.cdg_batch_step(uw, args.warmup, use_graph=False)
    del uw
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    launches0 = batch.cdg_batch_launch_count()
    torch.cuda.synchronize()
    ev[0].record(stream)
    batch.cdg_batch_step(ub, args.steps, persistent=True)
    ev[1].record(stream)
    torch.cuda.synchronize()
    st = batch.cdg_batch_check_status()
    if st != G.CDG_OK:
        raise G.CdgError(st, "batched steps")
    launches = batch.cdg_batch_launch_count() - launches0
    ms_b = ev[0].elapsed_time(ev[1])
    bps, pgrid = batch.cdg_batch_grid()
    # the same steps as per-phase launches captured in a graph
    ug = [u.clone() for u in u0]
    batch.cdg_batch_step(ug, 1, use_graph=True)  # capture a 1-step graph once (warm-up)
    ug = [u.clone() for u in u0]
    torch.cuda.synchronize()
    evg = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    evg[0].record(stream)
    for _ in range(args.steps):
        batch.cdg_batch_step(ug, 1, use_graph=True)
    evg[1].record(stream)
    torch.cuda.synchronize()
    ms_g = evg[0].elapsed_time(evg[1])
    # per-instance launches of the same kernels on the same stream
    ui = [u.clone() for u in u0]
    for c, u in zip(ctxs, ui):
        c.cdg_step_async(u, 0.0, 0.0, 1)
    torch.cuda.synchronize()
    ui = [u.clone() for u in u0]
    torch.cuda.synchronize()
    ev[2].record(stream)
    for c, u in zip(ctxs, ui):
        c.cdg_step_async(u, 0.0, 0.0, args.steps)
    ev[3].record(stream)
    torch.cuda.synchronize()
    ms_i = ev[2].elapsed_time(ev[3])
    diff = max(((a - b).abs().sum() / b.abs().sum()).item() for a, b in zip(ub, ui))
    same = all(torch.equal(a, b) for a, b in zip(ub, ug))  # persistent vs per-phase, same tile height
    # the single-mesh kernels use 4-row tiles: bitwise equal to the batch when it does too
    same_pi = all(torch.equal(a, b) for a, b in zip(ub, ui)) if rows == 4 else None
    line = {"metric": "FP64 DOF-updates/s per RK stage, batched 2D Euler Q2 (256 meshes)", "impl": "ours",
            "workload": f"batched_{args.count}_seed{args.seed}", "value": 3.0 * dof * args.steps / (ms_b * 1e-3),
            "unit": UNIT, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b / args.steps,
            "dof": dof, "sizes": sorted({q.n for q in insts}), "rows": rows, "gpu_launches": launches,
            "persistent_grid": {"blocks_per_sm": bps, "blocks": pgrid},
            "graph_per_phase": {"value": 3.0 * dof * args.steps / (ms_g * 1e-3), "ms_per_step": ms_g / args.steps,
                                "launches_per_step": 11},
            "per_instance": {"value": 3.0 * dof * args.steps / (ms_i * 1e-3), "ms_per_step": ms_i / args.steps,
                             "launches_per_step": 12 * args.count},
            "speedup_vs_per_instance": ms_i / ms_b, "speedup_vs_graph_per_phase": ms_g / ms_b,
            "identical_persistent_vs_per_phase": same, "identical_vs_per_instance": same_pi,
            "max_rel_l1_batched_vs_per_instance": diff,
            "dtype": "f64", "data": "synthetic"}
    print(json.dumps(line), flush=True)


# central-difference step sizes of the adjoint's finite-difference check
FD_STEPS = (1e-6, 1e-7, 1e-8, 1e-9, 1e-10)


def run_adjoint(args, ws, rank, local):
    """Isentropic vortex (strength 5) on uniform flow (1, 1), [0,10]^2 periodic,
    256^2 Q^2, plus a seeded 1e-3 Gaussian perturbation of every modal
    coefficient; loss 0.5 ||rho(T) - rho_target||^2 over the rho modal
    coefficients of both meshes, rho_target from the unperturbed run; gradient
    w.r.t. the initial coefficients through all stages and OE steps with
    sqrt(steps) checkpoints.  Reports adj/fwd = t(forward with checkpoints +
    backward) / t(plain forward) and central finite differences on seeded
    directions."""
    import torch
    from paper_2503_12473_gb300 import oecdg as G
    from paper_2503_12473_gb300 import workloads as W
    from paper_2503_12473_gb300.autograd import rollout

    torch.cuda.set_device(local)
    G.load()
    n, nsteps = args.n if args.n != 1024 else 256, args.steps
    w = W.vortex_2d(n=n)
    stream = torch.cuda.Stream()
    ctx = G.Context(G.desc_from_workload(w), stream=stream)
    with torch.cuda.stream(stream):
        base = ctx.project(w.u0)
        target = base.clone()
        ctx.cdg_step_async(target, 0.0, 0.0, nsteps)
        target = target[:, 0].clone()
        u0 = base + torch.from_numpy(W.perturbation(tuple(base.shape), args.seed + 1, 1e-3)).cuda()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        # warm-up of both paths (module load, adjoint scratch allocation)
        wu = u0.clone().requires_grad_(True)
        (rollout(wu, ctx, max(args.warmup, 1)) ** 2).sum().backward()
        del wu
        # plain forward
        x = u0.clone()
        torch.cuda.synchronize()
        ev[0].record(stream)
        ctx.cdg_step_async(x, 0.0, 0.0, nsteps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        t_fwd = ev[0].elapsed_time(ev[1])
        # forward with checkpoints + backward
        ui = u0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        ev[2].record(stream)
        uT = rollout(ui, ctx, nsteps)
        loss = 0.5 * ((uT[:, 0] - target) ** 2).sum()
        loss.backward()
        ev[3].record(stream)
        torch.cuda.synchronize()
        t_adj = ev[2].elapsed_time(ev[3])
        grad = ui.grad.detach()

        def L(v):
            y = v.clone()
            ctx.cdg_step_async(y, 0.0, 0.0, nsteps)
            return 0.5 * ((y[:, 0] - target) ** 2).sum().item()

        gen = torch.Generator(device="cpu").manual_seed(args.seed + 64)
        fd = []
        for _ in range(args.fd_dirs):
            d = torch.randn(tuple(u0.shape), generator=gen, dtype=torch.float64).cuda()
            an = (grad * d).sum().item()
            row = {"analytic": an}
            for h in FD_STEPS:
                f = (L(u0 + h * d) - L(u0 - h * d)) / (2 * h)
                row[f"rel_err_h{h:.0e}"] = abs(an - f) / max(abs(f), 1e-300)
            fd.append(row)
    # per step size, the worst direction; the best step balances the kinks of
    # the max operations (error ~ h) against rounding in L (error ~ eps / h)
    fd_max = {f"{h:.0e}": max(r[f"rel_err_h{h:.0e}"] for r in fd) for h in FD_STEPS} if fd else {}
    line = {"metric": "adjoint cost adj/fwd, 2D Euler Q2 vortex", "workload": f"euler_2d_vortex_q2_{n}",
            "steps": nsteps, "checkpoints": math.ceil(math.sqrt(nsteps)), "ms_forward": t_fwd,
            "ms_forward_checkpointed_plus_backward": t_adj, "adj_over_fwd": t_adj / t_fwd,
            "loss": loss.item(), "fd": fd,
            "fd_max_rel_err_by_h": fd_max,
            "fd_best": min(fd_max.items(), key=lambda kv: kv[1]) if fd_max else None,
            "dtype": "f64", "data": "synthetic"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024, help="cells per direction (the workload is 1024)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="riemann", choices=["riemann", "batched", "adjoint", "steady-wave", "advection-1d",
                                                       "shu-osher"],
                    help="riemann: the metric's workload (default); batched: 256 uneven meshes; "
                         "adjoint: gradient of the vortex loss (cost and finite-difference check); "
                         "steady-wave: the degree-generic 2D kernels on the smooth Euler test of Table 4; "
                         "advection-1d, shu-osher: time to solution of the 1D workloads")
    ap.add_argument("--k", type=int, default=3, help="steady-wave: degree 1..3")
    ap.add_argument("--basis", default="P", choices=["P", "Q"], help="steady-wave: P^k or Q^k")
    ap.add_argument("--fd-dirs", type=int, default=4)
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    ws, rank, local = init_dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batched":
        run_batched(args, ws, rank, local)
    elif args.workload == "adjoint":
        run_adjoint(args, ws, rank, local)
    elif args.workload == "steady-wave":
        run_generic(args, ws, rank, local)
    elif args.workload in ("advection-1d", "shu-osher"):
        run_time_to_solution(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
