"""Stress run: 2048x2048 intervals, Re = 30000, mixed precision, dt by the
rule, with checkpoints every `--every` steps, each one checked with the FP64
CPU oracle at full resolution:

  * the checkpoint round-trips (lc_save / lc_load restore the same bits);
  * Thom's wall vorticity (Eq. (25)) recomputed by the oracle from the saved
    psi equals the saved walls to 1e-6 relative;
  * the saved pair solves the compact Poisson problem: the oracle's relative
    residual ||f - L_h psi|| / ||f|| of (psi, omega), with f assembled from
    the saved omega (walls included, i.e. lagged as in the step), is <= 1e-6;
  * one FP64 oracle step from the checkpoint against one mixed GPU step from
    the same state: <= 1e-6 relative in psi and omega;
  * the steady-state monitors max|d omega|/dt, RES_psi, RES_omega.
The fields restricted to 257^2 by injection (stride 8) are saved as .npy.

    python -m tests.studies.stress_study --steps 20000 --every 5000 --out DIR [--summary stress.json]
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=2048)
    ap.add_argument("--Re", type=float, default=30000.0)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=5000)
    ap.add_argument("--out", default="stress_out")
    ap.add_argument("--summary", default=None, help="also write the JSON summary to this file")
    args = ap.parse_args()
    import torch

    import oracle
    from paper_0809_3098_gb300 import lc

    os.makedirs(args.out, exist_ok=True)
    torch.cuda.set_device(0)
    N, Re = args.N, args.Re
    cav = lc.Cavity(N, Re, precision=lc.LC_PREC_MIXED, monitor=1)
    dt = cav.params["dt"]
    records = []
    done = 0
    t0 = time.perf_counter()
    while done < args.steps:
        n = min(args.every, args.steps - done)
        cav.step(n)
        cav.synchronize()
        done += n
        mon = cav.monitor()
        path = os.path.join(args.out, f"ck_{done}.bin")
        cav.save(path)
        psi, om = cav.psi(), cav.omega()
        # round trip
        chk = lc.Cavity(N, Re, precision=lc.LC_PREC_MIXED)
        chk.load(path)
        roundtrip = bool(np.array_equal(chk.psi(), psi) and np.array_equal(chk.omega(), om))
        # Thom walls from the saved psi
        w_thom = oracle.thom(N, psi, om)
        thom_err = rel(w_thom, om)
        # Poisson residual of the saved pair, f from the saved omega
        f = oracle.poisson_rhs(N, oracle.OP_COMPACT, om)
        r = oracle.residual(N, oracle.OP_COMPACT, psi, f)
        pois_rel = float(np.linalg.norm(r) / np.linalg.norm(f))
        # one oracle FP64 step vs one GPU mixed step from the checkpoint
        ref = oracle.Cavity(N, Re, dt, 1e-10)
        ref.set_state(psi, om)
        ts = time.perf_counter()
        ref.step(1)
        t_oracle = time.perf_counter() - ts
        chk.step(1)
        step_err = {"psi": rel(chk.psi(), ref.psi()), "omega": rel(chk.omega(), ref.omega())}
        chk.close()
        ref.close()
        np.save(os.path.join(args.out, f"psi257_{done}.npy"), psi[::8, ::8])
        np.save(os.path.join(args.out, f"omega257_{done}.npy"), om[::8, ::8])
        rec = {"step": done, "t": done * dt, "max_domega_dt": mon[0], "RES_psi": mon[1], "RES_omega": mon[2],
               "roundtrip_bitwise": roundtrip, "thom_rel_err": thom_err, "poisson_rel_residual": pois_rel,
               "one_step_vs_oracle": step_err, "oracle_step_seconds": t_oracle,
               "psi_min": float(psi.min()), "gpu_seconds_so_far": time.perf_counter() - t0}
        records.append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
        os.remove(path)
    text = json.dumps({"command": "python -m tests.studies.stress_study " + " ".join(sys.argv[1:]),
                       "N": N, "Re": Re, "dt": dt, "steps": args.steps, "checkpoints": records})
    if args.summary:
        with open(args.summary, "w") as f:
            f.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
