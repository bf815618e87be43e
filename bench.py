#!/usr/bin/env python
"""Benchmark of the lid-driven-cavity SSPRK(5,4) step.

Metric: grid-point-stage updates per second = (N-1)^2 interior nodes x 5
Runge-Kutta stages x steps / time.  A "step" is one full SSPRK(5,4) step of
the default workload: 1024x1024 intervals, Re = 10000, lid u = 1, dt =
0.25 min(h, Re h^2/4), Poisson relative residual 1e-10, FP64, compact
fourth-order Poisson operator, starting from rest (synthetic, deterministic).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fp64-1024|fp64-128|fp64-4096] [--precision fp64|mixed]
                  [--eager] [--no-cpu-baseline] [--no-e2e] [--no-variants]

--precision mixed runs the same workload with FP32 multigrid V-cycles
inside FP64 residual, refinement, L(omega), Thom and stage accumulation (the
library's default; option rhs64 = 0 would take L(omega) from FP32 shadows).  --eager launches the step's kernels one by one (the V-cycle
loop driven from the host) so that a profiler can attribute them; it is
slower and only for profiling.

Our arm times K steps with CUDA events on the context's stream, flushing L2
(a 256 MiB write) between timed steps, and prints one JSON line with the
roofline of the dominant kernel, the CPU oracle timed on this host beside it,
the end-to-end rate through the C ABI with host buffers, the SM clocks seen
during the timed region and the kernel launch count.  The reference arm
(--impl reference) times the plain FP64 CPU oracle on the host cores on the
same workload.  Under torchrun (N > 1) every rank advances its own cavity
(independent replicas, no data exchange; weak scaling) and the slowest rank's
time is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_0809_3098_gb300.workloads import CAVITY_128_RE1000, CAVITY_1024_RE10000, Workload  # noqa: E402

# fp64-4096 is a profiling case: its fields (134 MB each) exceed the 126 MB L2.
WORKLOADS = {"fp64-1024": CAVITY_1024_RE10000, "fp64-128": CAVITY_128_RE1000,
             "fp64-4096": Workload("cavity-4096-Re10000-fp64", 4096, 10000.0, 10)}
# Multigrid smoothing schedule V(nu1, nu2) and smoother relaxation beta of the
# single-cavity runs (the library's defaults, set explicitly so that the
# kernel counts below match and the oracle runs the same schedule).
SCHEDULE = {"nu1": 2, "nu2": 1, "beta": 1.1}
METRIC = "grid-point-stage updates/s"
UNIT = "updates/s"
L2_FLUSH_BYTES = 256 << 20
CPU_SAMPLE_SECONDS = 8.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch32"], default="fp64-1024")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--eager", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--opt", action="append", default=[], metavar="KEY=VALUE",
                    help="an lc_set_option key for the single-cavity contexts (profiling; repeatable)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# FP64 peak of the part: 152 SMs x 2 FP64 FMA per clock per SM x 2 flops x
# the SM clock.  At the 2070 MHz maximum this is 1.26 TFLOP/s, the part's
# nominal FP64 rate.
SMS = 152
FP64_FMA_PER_CLK_PER_SM = 2


def fp64_peak_tflops(mhz: float) -> float:
    return SMS * FP64_FMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

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
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def host_cores() -> int:
    """Cores this process may run on (the affinity mask where the OS has one)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_rate(wl: Workload, budget_s: float, threads: int = 1):
    """Times the plain C oracle from rest on this host with `threads` OpenMP
    threads (the same bits for any count) for at least one step and until
    budget_s has passed.  Returns (updates/s, steps, s)."""
    import oracle

    oracle.set_threads(threads)
    try:
        cav = oracle.Cavity(wl.N, wl.Re, wl.dt, wl.tol, **SCHEDULE)
        steps, t0 = 0, time.perf_counter()
        while True:
            cav.step(1)
            steps += 1
            el = time.perf_counter() - t0
            if el >= budget_s or steps >= 1000:
                break
        cav.close()
    finally:
        oracle.set_threads(1)
    return wl.interior_nodes * 5 * steps / el, steps, el


def run_reference(args, wl: Workload):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    cores = host_cores()
    oracle.set_threads(cores)
    cav = oracle.Cavity(wl.N, wl.Re, wl.dt, wl.tol, **SCHEDULE)
    cav.step(args.warmup)
    t0 = time.perf_counter()
    cav.step(args.steps)
    el = time.perf_counter() - t0
    oracle.set_threads(1)
    value = wl.interior_nodes * 5 * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed SSPRK(5,4) steps after {args.warmup} from rest, "
                                   f"{wl.N}x{wl.N}, plain C FP64, OpenMP over the independent loops on "
                                   f"{cores} threads (reductions serial; the same bits as one thread)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_of(wl: Workload, gpus: int, precision: str = "fp64") -> dict:
    name = wl.name if precision == "fp64" else wl.name.replace("-fp64", "-mixed")
    return {"workload": name, "N": wl.N, "Re": wl.Re, "dt": wl.dt, "tol": wl.tol, "op": wl.op,
            "precision": precision, "schedule": f"V({SCHEDULE['nu1']},{SCHEDULE['nu2']}), beta {SCHEDULE['beta']}",
            "start": "rest (psi = omega = 0)",
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": "replicas" if gpus > 1 else "single"}


FP32_FMA_PER_CLK_PER_SM = 128


def nvtx(torch, name):
    """Opens (name) or closes (None) an NVTX range; a no-op where NVTX is missing."""
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time: all-reduce MAX over the process group (any backend)."""
    import torch

    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, max_ms: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank in at most max_ms."""
    return world * units_per_rank / (max_ms * 1e-3)

# Kernels lc_bench_kernel can time (its kernel id), and how many launches of
# each a step makes (c = V-cycles in the step's five solves, nu = nu1 + nu2).
KERNELS = {
    "fp64": [(0, "k_smooth_colour<double,compact,relaxed> (fine level, one colour phase, beta != 1)",
              lambda c, nu: 4 * nu * c),
             (1, "k_rhs_stage (fused L(omega) + stage combination)", lambda c, nu: 5),
             (2, "k_residual_restrict<double,compact> (fine level)", lambda c, nu: c)],
    "mixed": [(0, "k_down<float,compact> (fine level: FP32 pre-smoothing + residual + restriction)", lambda c, nu: c),
              (1, "k_rhs_stage (FP64 L(omega) + stage combination; option rhs64, the default)", lambda c, nu: 5),
              (2, "k_residual64_to32<compact> (FP64 residual, rounded to FP32)", lambda c, nu: c + 5),
              (3, "k_up<float,compact> (fine level: FP32 post-smoothing + FP64 psi += e)", lambda c, nu: c)],
}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per interior
# node of one launch, from one ncu capture of each kernel at 1024^2 with the
# step's arguments; a launch's traffic is this figure times its interior
# nodes (the kernels read and write every node once per launch, so the
# traffic grows with the node count).  A kernel without a capture of its
# current code reports null.
#   k_smooth_colour<double,compact>: 12,728,576 B per launch at 1024^2 over
#   1023^2 interior nodes = 12.163 B per node (12 B algorithmic); its
#   relaxed form (beta != 1, the default): 12,571,648 B = 12.01 B per node;
#   k_rhs_stage (stage 2): 25,440,768 B = 24.31 B per node (32 B algorithmic;
#   its output stays in L2 at this size);
#   k_residual64_to32: 16,930,560 B = 16.18 B per node (20 B algorithmic);
#   k_down<float> (110x22): 4,341,504 B = 4.15 B per node;
#   k_up<float> (110x22): 18,192,384 B = 17.38 B per node.
TRAFFIC_PER_NODE = {
    "k_smooth_colour<double,compact> (fine level, one colour phase)": 12728576 / 1023 ** 2,
    "k_smooth_colour<double,compact,relaxed> (fine level, one colour phase, beta != 1)": 12571648 / 1023 ** 2,
    "k_rhs_stage (fused L(omega) + stage combination)": 25440768 / 1023 ** 2,
    "k_rhs_stage (FP64 L(omega) + stage combination; option rhs64, the default)": 25440768 / 1023 ** 2,
    "k_residual64_to32<compact> (FP64 residual, rounded to FP32)": 16930560 / 1023 ** 2,
    "k_down<float,compact> (fine level: FP32 pre-smoothing + residual + restriction)": 4341504 / 1023 ** 2,
    "k_up<float,compact> (fine level: FP32 post-smoothing + FP64 psi += e)": 18192384 / 1023 ** 2,
}
TRAFFIC_MEASURED_AT = 1024  # the per-node figures hold where the fields fit L2 as at 1024^2


def roofline(lc, cav, precision: str, cycles_per_step: float, clocks: dict) -> dict:
    """Times each fine-level kernel of the step (lc_bench_kernel, CUDA events on
    the context stream, the same arguments as in the step) and reports the one
    with the largest share of the step against whichever peak binds it."""
    hbm, max_mhz, src = peaks()
    mhz = clocks.get("sm_mhz") or max_mhz
    p64 = fp64_peak_tflops(mhz)
    p32 = SMS * FP32_FMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12
    rows = []
    nu = SCHEDULE["nu1"] + SCHEDULE["nu2"]
    for kid, name, count in KERNELS[precision]:
        ms, nbytes, f64, f32 = lc.lc_bench_kernel(cav.handle, kid, 100)
        share_ms = ms * count(cycles_per_step, nu)
        fr = {"hbm": nbytes / (ms * 1e-3) / 1e9 / hbm, "alu64": f64 / (ms * 1e-3) / 1e12 / p64,
              "alu32": f32 / (ms * 1e-3) / 1e12 / p32}
        rows.append((share_ms, kid, name, ms, nbytes, f64, f32, fr))
    share_ms, kid, name, ms, nbytes, f64, f32, fr = max(rows)
    bound = max(fr, key=fr.get)
    if bound == "hbm":
        roof = {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_source": f"{src} copy bandwidth (MEASURED_PEAKS.json), of {src}"}
    else:
        fl, pk = (f64, p64) if bound == "alu64" else (f32, p32)
        roof = {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": pk, "unit": "TFLOP/s",
                "peak_source": (f"derived: {SMS} SMs x "
                                f"{FP64_FMA_PER_CLK_PER_SM if bound == 'alu64' else FP32_FMA_PER_CLK_PER_SM} "
                                f"{'FP64' if bound == 'alu64' else 'FP32'} FMA/clk x 2 flop x {mhz:.0f} MHz "
                                f"(median SM clock under load)")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    per_node = TRAFFIC_PER_NODE.get(name) if cav.N == TRAFFIC_MEASURED_AT else None
    roof["traffic"] = round(per_node * (cav.N - 1) ** 2) if per_node is not None else None
    roof["kernel"] = name
    roof["kernel_ms"] = ms
    roof["launches_per_step"] = {k: f for k, _, f in KERNELS[precision]}[kid](cycles_per_step, nu)
    roof["algorithmic_bytes"] = nbytes
    roof["fp64_flops"] = f64
    roof["fp32_flops"] = f32
    roof["fractions"] = fr
    roof["all_kernels_ms"] = {r[2]: r[3] for r in sorted(rows, key=lambda r: r[1])}
    return roof


def parse_opts(pairs) -> dict:
    """--opt KEY=VALUE pairs as lc_set_option arguments."""
    out = {}
    for p in pairs:
        k, _, v = p.partition("=")
        out[k.strip()] = float(v)
    return out


def timed_run(lc, torch, dist, wl: Workload, precision: str, steps: int, warmup: int, eager: bool, world: int,
              sample_clocks: int | None, extra: dict | None = None):
    """W warm-up steps, then K steps each bracketed by CUDA events on the
    context's stream, with an L2 flush between them."""
    opts = {"op": lc.LC_OP_COMPACT, "precision": lc.LC_PREC_MIXED if precision == "mixed" else lc.LC_PREC_FP64,
            **SCHEDULE, **(extra or {})}
    if eager:
        opts["graph"] = 0
    cav = lc.Cavity(wl.N, wl.Re, wl.dt, wl.tol, **opts)
    stream = torch.cuda.current_stream()
    cav.step(warmup)
    cav.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    n_before = len(cav.cycle_log())
    sampler = None
    if sample_clocks is not None:
        sampler = ClockSampler(sample_clocks)
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    nvtx(torch, "timed_steps")  # lets a profiler select the timed launches
    for k in range(steps):
        flush.fill_(k & 0xFF)  # evicts the previous step's working set from L2
        ev[k][0].record(stream)
        cav.step(1)
        ev[k][1].record(stream)
    nvtx(torch, None)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else {}
    cav.synchronize()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist if world > 1 else None, "cuda")
    cycles = cav.cycle_log()[n_before:]
    per_step_fixed, per_cycle = lc.lc_launch_stats(cav.handle)
    return {
        "cav": cav, "total_ms": total_ms, "wall_ms": wall * 1e3, "clocks": clocks,
        "cycles": cycles, "launches": int(steps * per_step_fixed + per_cycle * int(cycles.sum())),
        "value": job_rate(world, wl.interior_nodes * 5 * steps, total_ms),
    }


def mixed_bytes_per_node(cycles_per_step: float, rhs64: bool = True) -> float:
    """Algorithmic DRAM bytes per interior node of one mixed-precision step
    (each array element read or written once per kernel):
    L(omega) + stage combination over the five stages: in FP64 (option
    rhs64, the default) 24+32+40+48+32 = 176 B, from the FP32 shadows
    28+36+44+52+36 = 196 B plus the FP32 shadow of psi after each solve
    5 x 12 B; Poisson right-hand side 5 x 16 B; the first FP64 residual of
    each solve 5 x 20 B; per refinement cycle: fine-level FP32 pre-smoothing
    tile 9 B (r32 in, e32 out, coarse g out), post-smoothing tile + psi64 += e
    25 B (e32, r32, coarse e in; psi64 in and out), FP64 residual 20 B
    (psi64, g64 in; r32 out), and the coarser levels' tiles, 22 B per coarse
    node summed over levels (22/4 + 22/16 + ...)."""
    per_cycle = 9.0 + 25.0 + 20.0 + 22.0 / 3.0
    stage = 176.0 if rhs64 else 196.0 + 60.0
    return stage + 80.0 + 100.0 + cycles_per_step * per_cycle


def run_batch(lc, torch, args, world: int, eager: bool = False) -> dict:
    import numpy as np

    from paper_0809_3098_gb300.workloads import batch_cavities

    cav = batch_cavities(32, seed=0)
    Ns, Res = [n for n, _ in cav], [r for _, r in cav]
    b = lc.Batch(Ns, Res, graph=0 if eager else 1)
    b.step(1)
    b.synchronize()
    schedule = b.autotune_schedule(steps=2)
    shapes = b.autotune(reps=3)
    b.step(max(args.warmup - 1, 0))
    b.synchronize()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    n_before = [len(b.cycle_log(c)) for c in range(b.count)]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    nvtx(torch, "timed_steps")
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        b.step(1)
        ev[k][1].record(stream)
    nvtx(torch, None)
    torch.cuda.synchronize()
    b.synchronize()
    total_ms = sum(a.elapsed_time(c) for a, c in ev)
    nodes = [(n - 1) ** 2 for n in Ns]
    cyc = [b.cycle_log(c)[n_before[c]:] for c in range(b.count)]
    per_step_cycles = [x.sum() / args.steps for x in cyc]
    nbytes = sum(n * mixed_bytes_per_node(c) for n, c in zip(nodes, per_step_cycles)) * args.steps
    hbm, _, src = peaks()
    gbs = nbytes / (total_ms * 1e-3) / 1e9
    b.close()
    return {
        "value": world * sum(nodes) * 5 * args.steps / (total_ms * 1e-3), "unit": UNIT,
        "ms_per_step": total_ms / args.steps, "cavities": len(Ns), "interior_nodes": sum(nodes),
        "N": Ns, "Re": [round(r, 1) for r in Res], "vcycles_per_solve": float(np.mean(np.concatenate(cyc))) / 1.0,
        "tile_shapes_autotuned": shapes, "schedule_autotuned": {"nu1": schedule[0], "nu2": schedule[1]},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "scope": "whole step: algorithmic bytes of every kernel / step time",
                     "peak_source": f"{src} copy bandwidth (MEASURED_PEAKS.json)"},
        "l2": "flushed between timed steps (256 MiB write); the batch's arrays (~1 GB) exceed L2",
    }


def run_sor(lc, torch, wl: Workload) -> dict:
    """Throughput of the lexicographic SOR kernel (Eq. (15) in its own order,
    16 sweeps per launch) on the workload's grid: node updates per second."""
    cav = lc.Cavity(wl.N, wl.Re, sor_sweeps=16, beta=1.5)
    cav.step(1)
    cav.synchronize()
    reps = 3
    r = lc.lc_bench_kernel(cav.handle, 3, reps)
    cav.close()
    ms = r[0]
    upd = 16 * (wl.N - 1) ** 2
    return {"value": upd / (ms * 1e-3), "unit": "node updates/s", "ms_per_16_sweeps": ms,
            "fp64_tflops": r[2] / (ms * 1e-3) / 1e12,
            "note": "one thread block (the sweep order is sequential beyond a wavefront); not a step rate"}


def run_ours(args, wl: Workload):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_0809_3098_gb300 import lc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    extra = parse_opts(args.opt)
    r = timed_run(lc, torch, dist, wl, args.precision, args.steps, args.warmup, args.eager, world, local, extra)
    cav = r["cav"]
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic", "config": config_of(wl, world, args.precision),
    }
    line["config"]["wall_ms_timed_region"] = r["wall_ms"]
    line["config"]["vcycles_per_solve"] = float(r["cycles"].mean()) if len(r["cycles"]) else None
    if args.eager:
        line["config"]["launch"] = "eager (profiling)"
    if extra:
        line["config"]["options"] = extra
    line["gpu_launches"] = r["launches"]
    line["clocks"] = r["clocks"]

    cyc_per_step = float(r["cycles"].sum()) / max(args.steps, 1)
    state = (cav.psi(), cav.omega())
    line["roofline"] = roofline(lc, cav, args.precision, cyc_per_step, r["clocks"])

    # --- end to end through the C ABI with host buffers (pinned)
    if not args.no_e2e:
        n = (wl.N + 1) ** 2
        hp = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy().reshape(wl.N + 1, wl.N + 1)
        hw = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy().reshape(wl.N + 1, wl.N + 1)
        hp[:], hw[:] = state
        e2e_steps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            cav.set_state(hp, hw)
            cav.step(1)
            lc._check(lc.lc_get_psi(cav.handle, hp), "lc_get_psi")
            lc._check(lc.lc_get_omega(cav.handle, hw), "lc_get_omega")
        e2e_s = time.perf_counter() - t0
        line["e2e"] = {"value": world * wl.interior_nodes * 5 * e2e_steps / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 2 * 8 * n,
                       "steps": e2e_steps, "api": "lc_set_state + lc_step(1) + lc_get_psi + lc_get_omega"}
    cav.close()

    # --- the mixed-precision form of the same workload, and its error against this FP64 run
    if not args.no_variants and args.precision == "fp64" and not args.eager:
        m = timed_run(lc, torch, dist, wl, "mixed", args.steps, args.warmup, False, world, None)
        mc = m["cav"]
        ep = float(np.abs(mc.psi() - state[0]).max() / np.abs(state[0]).max())
        ew = float(np.abs(mc.omega() - state[1]).max() / np.abs(state[1]).max())
        mcyc = float(m["cycles"].sum()) / max(args.steps, 1)
        line["variants"] = {"mixed": {
            "value": m["value"], "unit": UNIT, "ms_per_step": m["total_ms"] / args.steps,
            "speedup_vs_fp64": m["value"] / r["value"], "vcycles_per_solve": float(m["cycles"].mean()),
            "gpu_launches": m["launches"],
            "rel_err_vs_fp64": {"psi": ep, "omega": ew, "after_steps": args.warmup + args.steps},
            "roofline": roofline(lc, mc, "mixed", mcyc, r["clocks"]),
        }}
        mc.close()

    # --- the batched form: 32 cavities of uneven N and Re in one graph launch per step
    if not args.no_variants and args.precision == "fp64" and not args.eager:
        line["variants"]["batch32_mixed"] = run_batch(lc, torch, args, world)

    # --- the paper's own solver: lexicographic SOR sweeps (wavefront kernel, one block)
    if not args.no_variants and args.precision == "fp64" and not args.eager:
        line["variants"]["sor_lex_sweeps"] = run_sor(lc, torch, wl)

    # --- CPU oracle on this host (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        rate, steps, el = cpu_oracle_rate(wl, CPU_SAMPLE_SECONDS, cores)
        rate1, steps1, el1 = cpu_oracle_rate(wl, CPU_SAMPLE_SECONDS, 1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {steps} SSPRK(5,4) steps from rest of the same workload "
                                          f"({el:.1f} s), plain C FP64, OpenMP over the independent loops "
                                          f"(colour phases, stencils, transfers, stage combination; reductions "
                                          f"serial) on {cores} threads",
                                "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                                  "sample": f"first {steps1} steps from rest ({el1:.1f} s), "
                                                            f"one thread"}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch_only(args):
    """--workload batch32: the 32-cavity batch alone (a profiling case; with
    --eager its kernels are launched one by one so that ncu can see them)."""
    import torch

    from paper_0809_3098_gb300 import lc

    torch.cuda.set_device(0)
    r = run_batch(lc, torch, args, 1, eager=args.eager)
    line = {"metric": METRIC, "value": r.pop("value"), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "batch32-mixed", "launch": "eager (profiling)" if args.eager else "graph"},
            "roofline": r.pop("roofline"), "batch": r}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.workload == "batch32":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "batch32 is a profiling workload of ours only"}))
            return 0
        return run_batch_only(args)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
