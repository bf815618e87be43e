"""Precision study: the mixed-precision step against the FP64 step on the
lid-driven cavity, 1024x1024 intervals, Re in {5000, 10000, 20000, 30000},
dt by the rule 0.25 min(h, Re h^2 / 4), Poisson tol 1e-10, from rest.

Both runs use the CUDA library; the FP64 path is itself held to the plain
FP64 oracle at 1e-10 by the parity tests.  Reported per Re: the relative
max-norm error max|x - x_fp64| / max|x_fp64| of psi, omega, the vertical
centreline u(y) at x = 1/2 and the horizontal centreline v(x) at y = 1/2
(central differences of psi, Eq. (22); wall values by the boundary
conditions), and each path's time per step.  The mixed runs go through the
batched engine (all Re in one launch per step), which gives the bits of
single-cavity mixed runs, once in the default form (L(omega) in FP64, option
rhs64 = 1; FP32 multigrid corrections) and once with L(omega) in FP32 from
the FP32 shadows of psi and omega (rhs64 = 0).

    python -m tests.studies.precision_study --steps 20000 [--N 1024] [--out precision.json]
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def centrelines(psi: np.ndarray):
    N = psi.shape[0] - 1
    h = 1.0 / N
    m = N // 2
    u = np.zeros(N + 1)
    u[1:N] = (psi[2:, m] - psi[:-2, m]) / (2 * h)  # u(y) at x = 1/2, psi[j, i]
    u[N] = 1.0
    v = np.zeros(N + 1)
    v[1:N] = -(psi[m, 2:] - psi[m, :-2]) / (2 * h)  # v(x) at y = 1/2
    return u, v


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--Re", type=float, nargs="*", default=[5000.0, 10000.0, 20000.0, 30000.0])
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch

    from paper_0809_3098_gb300 import lc

    torch.cuda.set_device(0)
    out = {"command": "python -m tests.studies.precision_study " + " ".join(sys.argv[1:]),
           "N": args.N, "steps": args.steps, "tol": 1e-10, "results": []}
    t0 = time.perf_counter()
    batch = lc.Batch([args.N] * len(args.Re), args.Re)
    batch.step(args.steps)
    batch.synchronize()
    t_mixed = time.perf_counter() - t0
    # the same with L(omega) in FP32 (rhs64 = 0): separates the error of the
    # FP32 stencils from that of the FP32 multigrid corrections
    t0 = time.perf_counter()
    batch32 = lc.Batch([args.N] * len(args.Re), args.Re, rhs64=0)
    batch32.step(args.steps)
    batch32.synchronize()
    t_mixed32 = time.perf_counter() - t0
    for c, Re in enumerate(args.Re):
        t1 = time.perf_counter()
        ref = lc.Cavity(args.N, Re, monitor=1)
        monitors = []
        done = 0
        while done < args.steps:  # the steady-state monitors every 1000 steps
            n = min(1000, args.steps - done)
            ref.step(n)
            done += n
            m = ref.monitor()
            monitors.append({"step": done, "max_domega_dt": m[0], "RES_psi": m[1], "RES_omega": m[2]})
        ref.synchronize()
        t_fp64 = time.perf_counter() - t1
        p64, w64 = ref.psi(), ref.omega()
        pm, wm = batch.psi(c), batch.omega(c)
        pr, wr = batch32.psi(c), batch32.omega(c)
        u64, v64 = centrelines(p64)
        um, vm = centrelines(pm)
        ur, vr = centrelines(pr)
        row = {"Re": Re, "dt": ref.params["dt"], "t_end": ref.params["dt"] * args.steps,
               "rel_err": {"psi": rel(pm, p64), "omega": rel(wm, w64), "u_centre": rel(um, u64),
                           "v_centre": rel(vm, v64)},
               "rel_err_fp32_L": {"psi": rel(pr, p64), "omega": rel(wr, w64), "u_centre": rel(ur, u64),
                                  "v_centre": rel(vr, v64)},
               "psi_min": float(p64.min()), "fp64_ms_per_step": 1e3 * t_fp64 / args.steps,
               "fp64_monitors": monitors,
               "vcycles_per_solve": {"fp64": float(ref.cycle_log().mean()),
                                     "mixed": float(batch.cycle_log(c).mean()),
                                     "mixed_fp32_L": float(batch32.cycle_log(c).mean())}}
        out["results"].append(row)
        ref.close()
        print(json.dumps(row), file=sys.stderr, flush=True)
    n = len(args.Re)
    out["mixed_batch_ms_per_step"] = {"cavities": n, "default": 1e3 * t_mixed / args.steps,
                                      "fp32_L": 1e3 * t_mixed32 / args.steps}
    text = json.dumps(out)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
