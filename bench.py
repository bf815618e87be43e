#!/usr/bin/env python
"""Benchmark of the lid-driven-cavity SSPRK(5,4) step.

Metric: grid-point-stage updates per second = (N-1)^2 interior nodes x 5
Runge-Kutta stages x steps / time.  A "step" is one full SSPRK(5,4) step of
the default workload: 1024x1024 intervals, Re = 10000, lid u = 1, dt =
0.25 min(h, Re h^2/4), Poisson relative residual 1e-10, FP64, compact
fourth-order Poisson operator, starting from rest (synthetic, deterministic).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fp64-1024|fp64-128]

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
METRIC = "grid-point-stage updates/s"
UNIT = "updates/s"
L2_FLUSH_BYTES = 256 << 20
CPU_SAMPLE_SECONDS = 12.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="fp64-1024")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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


def cpu_oracle_rate(wl: Workload, budget_s: float):
    """Times the plain C oracle from rest on this host (single thread) for at
    least one step and until budget_s has passed.  Returns (updates/s, steps, s)."""
    import oracle

    cav = oracle.Cavity(wl.N, wl.Re, wl.dt, wl.tol)
    steps, t0 = 0, time.perf_counter()
    while True:
        cav.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 1000:
            break
    cav.close()
    return wl.interior_nodes * 5 * steps / el, steps, el


def run_reference(args, wl: Workload):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    cav = oracle.Cavity(wl.N, wl.Re, wl.dt, wl.tol)
    cav.step(args.warmup)
    t0 = time.perf_counter()
    cav.step(args.steps)
    el = time.perf_counter() - t0
    value = wl.interior_nodes * 5 * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} timed SSPRK(5,4) steps after {args.warmup} from rest, "
                                   f"{wl.N}x{wl.N}, plain C FP64, one thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_of(wl: Workload, gpus: int) -> dict:
    return {"workload": wl.name, "N": wl.N, "Re": wl.Re, "dt": wl.dt, "tol": wl.tol, "op": wl.op,
            "precision": wl.precision, "start": "rest (psi = omega = 0)",
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": "replicas" if gpus > 1 else "single"}


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

    cav = lc.Cavity(wl.N, wl.Re, wl.dt, wl.tol, op=lc.LC_OP_COMPACT)
    stream = torch.cuda.current_stream()
    cav.step(args.warmup)
    cav.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    n_before = len(cav.cycle_log())

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # evicts the previous step's working set from L2
        ev[k][0].record(stream)
        cav.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    cav.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    cycles = cav.cycle_log()[n_before:]
    per_step_fixed, per_cycle = lc.lc_launch_stats(cav.handle)
    launches = int(args.steps * per_step_fixed + per_cycle * int(cycles.sum()))

    updates = wl.interior_nodes * 5 * args.steps
    value = world * updates / (total_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(wl, world),
    }
    line["config"]["wall_ms_timed_region"] = wall * 1e3
    line["config"]["vcycles_per_solve"] = float(cycles.mean()) if len(cycles) else None
    line["gpu_launches"] = launches
    line["clocks"] = clocks

    # --- roofline of the dominant kernel: the fine-level smoother colour phase
    hbm, max_mhz, src = peaks()
    reps = 200
    k = lc.lc_bench_kernel(cav.handle, 0, reps)
    ms, nbytes, f64 = k[0], k[1], k[2]
    mhz_load = clocks.get("sm_mhz") or max_mhz
    p64 = fp64_peak_tflops(mhz_load)
    ach_tf = f64 / (ms * 1e-3) / 1e12
    ach_gbs = nbytes / (ms * 1e-3) / 1e9
    alu_frac, hbm_frac = ach_tf / p64, ach_gbs / hbm
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": ach_tf, "peak": p64, "unit": "TFLOP/s", "frac": alu_frac}
        roof["peak_source"] = (f"derived: {SMS} SMs x {FP64_FMA_PER_CLK_PER_SM} FP64 FMA/clk x 2 flop x "
                               f"{mhz_load:.0f} MHz (median SM clock under load)")
    else:
        roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm, "unit": "GB/s", "frac": hbm_frac,
                "peak_source": f"{src} copy bandwidth (MEASURED_PEAKS.json)"}
    roof["traffic"] = None
    roof["kernel"] = "k_smooth_colour<double,compact> (fine level, one colour phase)"
    roof["kernel_ms"] = ms
    roof["algorithmic_bytes"] = nbytes
    roof["fp64_flops"] = f64
    roof["hbm_frac"] = hbm_frac
    roof["alu_frac"] = alu_frac
    line["roofline"] = roof

    # --- end to end through the C ABI with host buffers (pinned)
    n = (wl.N + 1) ** 2
    hp = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy().reshape(wl.N + 1, wl.N + 1)
    hw = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy().reshape(wl.N + 1, wl.N + 1)
    hp[:] = cav.psi()
    hw[:] = cav.omega()
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        cav.set_state(hp, hw)
        cav.step(1)
        lc.lc_get_psi(cav.handle, hp)
        lc._check(lc.lc_get_omega(cav.handle, hw), "lc_get_omega")
    e2e_s = time.perf_counter() - t0
    line["e2e"] = {"value": world * wl.interior_nodes * 5 * e2e_steps / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 2 * 8 * n,
                   "steps": e2e_steps, "api": "lc_set_state + lc_step(1) + lc_get_psi + lc_get_omega"}

    # --- CPU oracle on this host (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, steps, el = cpu_oracle_rate(wl, CPU_SAMPLE_SECONDS)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {steps} SSPRK(5,4) steps from rest of the same workload "
                                          f"({el:.1f} s), plain C FP64, one thread"}
    if rank == 0:
        print(json.dumps(line))
    cav.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
