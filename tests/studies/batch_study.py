"""Batch study: the 32-cavity workload (N drawn from {256, 384, 512, 768,
1024}, Re log-uniform in [1000, 30000], seed 0) advanced for `--steps` steps
in one mixed-precision batch with the autotuned smoothing schedule and tile
shapes; the whole run's throughput, and for a few cavities (the smallest, the
largest and the one with the highest Re) the relative max-norm error against
an FP64 single-cavity run of the same steps, in psi, omega and the
centreline velocities.

    python -m tests.studies.batch_study --steps 5000 [--out batch.json]
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from tests.studies.precision_study import centrelines, rel  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--rhs64", type=int, default=None, help="L(omega) in FP64 (1, the default) or FP32 (0)")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch

    from paper_0809_3098_gb300 import lc
    from paper_0809_3098_gb300.workloads import batch_cavities

    torch.cuda.set_device(0)
    cav = batch_cavities(32, seed=0)
    Ns, Res = [n for n, _ in cav], [r for _, r in cav]
    opts = {} if args.rhs64 is None else {"rhs64": args.rhs64}
    b = lc.Batch(Ns, Res, **opts)
    schedule = b.autotune_schedule(steps=2)
    shapes = b.autotune(reps=3)
    nodes = sum((n - 1) ** 2 for n in Ns)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    b.step(args.steps)
    e1.record(s)
    e1.synchronize()
    b.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"command": "python -m tests.studies.batch_study " + " ".join(sys.argv[1:]),
           "steps": args.steps, "cavities": len(Ns), "interior_nodes": nodes, "N": Ns,
           "Re": [round(r, 1) for r in Res], "schedule": schedule,
           "tile_shapes": shapes, "rhs64": 1 if args.rhs64 is None else args.rhs64, "seconds": ms / 1e3,
           "updates_per_s": nodes * 5 * args.steps / (ms / 1e3), "checks": []}
    picks = sorted({int(np.argmin(Ns)), int(np.argmax(Ns)), int(np.argmax(Res))})
    for c in picks:
        t0 = time.perf_counter()
        ref = lc.Cavity(Ns[c], Res[c], nu1=schedule[0], nu2=schedule[1])
        ref.step(args.steps)
        ref.synchronize()
        p64, w64 = ref.psi(), ref.omega()
        pm, wm = b.psi(c), b.omega(c)
        u64, v64 = centrelines(p64)
        um, vm = centrelines(pm)
        row = {"cavity": c, "N": Ns[c], "Re": Res[c], "fp64_seconds": time.perf_counter() - t0,
               "rel_err": {"psi": rel(pm, p64), "omega": rel(wm, w64), "u_centre": rel(um, u64),
                           "v_centre": rel(vm, v64)}}
        out["checks"].append(row)
        ref.close()
        print(json.dumps(row), file=sys.stderr, flush=True)
    text = json.dumps(out)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
