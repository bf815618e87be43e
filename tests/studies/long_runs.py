"""Long runs towards steady state on single-cavity contexts (Cardoso & Bicudo,
arXiv:0809.3098, Sec. 3.2 monitors and the grid study of Sec. 4).

Every case is one context of the CUDA library.  The cases advance in turns,
`--every` steps at a time, until `--t-end`, `--max-seconds` or the paper's
steady-state thresholds (a case that meets them stops); after each
turn a case records the steady-state monitors of Eqs. (26)-(27) over its
last step (the library's "monitor" option: max |d omega| / dt, RES_psi,
RES_omega with 1/N read as 1/(N+1)) and psi at two probe nodes, so a
periodic flow shows as an oscillating probe.

    python -m tests.studies.long_runs floor  --out floor.json
        1024^2, Re 5000, dt 0.001 (the paper's Table 1): one mixed-precision
        context with L(omega) in FP64 from rest to --t-branch; there its state
        is installed in two contexts, L(omega) in FP64 (rhs64 = 1) and in FP32
        (rhs64 = 0), which both go on to --t-end.  Tests whether the FP32
        rounding of L(omega) puts a floor under the monitors.
    python -m tests.studies.long_runs coarse --out coarse.json
        The paper's coarse-grid cases (220^2 read as 224 intervals) at
        Re 10000 under several solver settings: multigrid solved to 1e-10 in
        mixed precision at the time steps --mg-dts (and in FP64 with --fp64), and the
        paper's own SOR iteration of Eq. (15) with a fixed budget of sweeps per
        stage (tol so large that every solve stops after one pass) at
        relaxation beta from the paper's 0.8 -> 0.1 range.
    python -m tests.studies.long_runs paper --out paper.json
        1024^2 at Re 10000, 20000, 30000, dt 0.001, mixed precision with
        L(omega) in FP64, from rest.

The output is one compact JSON object (monitor histories with 4 significant
digits) with the command line that made it.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from tests.studies.steady_study import vortex_census  # noqa: E402

PAPER_THRESHOLDS = {True: (1e-12, 1e-10), False: (1e-10, 1e-8)}  # keyed by Re <= 20000


def sig(x, n=4):
    return float(f"{x:.{n}g}")


class Case:
    def __init__(self, name, N, Re, dt, tol=1e-10, **opts):
        from paper_0809_3098_gb300 import lc

        self.name, self.N, self.Re = name, N, Re
        self.opts = dict(opts)
        self.cav = lc.Cavity(N, Re, dt, tol, monitor=1, **opts)
        self.dt = self.cav.params["dt"]
        self.steps = 0
        self.hist = []
        self.seconds = 0.0
        self.steady_at = None
        self.error = None  # set if the context reports an error (e.g. a non-finite state); the case stops
        self.thr = PAPER_THRESHOLDS[Re <= 20000]
        # probe nodes: the centre and a point in the bottom-right corner region
        self.probes = [(N // 2, N // 2), (int(round(0.9 * N)), int(round(0.1 * N)))]

    def advance(self, n):
        t0 = time.perf_counter()
        self.cav.step(n)
        m = self.cav.monitor()
        self.seconds += time.perf_counter() - t0
        self.steps += n
        psi = self.cav.psi()
        rec = {"t": sig(self.steps * self.dt, 6), "max_domega_dt": sig(m[0]), "RES_psi": sig(m[1]),
               "RES_omega": sig(m[2]), "cycles": int(m[3]),
               "probe": [sig(psi[j, i], 8) for i, j in self.probes], "psi_min": sig(psi.min(), 8)}
        self.hist.append(rec)
        if self.steady_at is None and m[1] < self.thr[0] and m[2] < self.thr[1]:
            self.steady_at = self.steps
        return rec

    def summary(self):
        h = self.hist
        if not h:
            return {"name": self.name, "N": self.N, "Re": self.Re, "dt": self.dt, "options": self.opts,
                    "error": self.error, "monitors": []}
        k = max(1, len(h) // 10)
        last, prev = h[-k:], h[-2 * k:-k] if len(h) >= 2 * k else h[:k]
        mx_last = max(r["max_domega_dt"] for r in last)
        mx_prev = max(r["max_domega_dt"] for r in prev)
        pr_last = [r["probe"][1] for r in last]
        if self.steady_at is not None:
            trend = "steady (paper thresholds met)"
        elif mx_last < 0.5 * mx_prev:
            trend = "decaying"
        else:
            trend = "not decaying"
        cyc = self.cav.cycle_log()
        return {"name": self.name, "N": self.N, "Re": self.Re, "dt": self.dt, "options": self.opts,
                "error": self.error, "steps": self.steps, "t_end": sig(self.steps * self.dt, 6), "seconds": round(self.seconds, 1),
                "ms_per_step": sig(1e3 * self.seconds / max(self.steps, 1)),
                "steady_at_step": self.steady_at, "thresholds": self.thr, "trend_last_tenth": trend,
                "max_domega_dt_last_tenth": [min(r["max_domega_dt"] for r in last), mx_last],
                "max_domega_dt_previous_tenth": [min(r["max_domega_dt"] for r in prev), mx_prev],
                "corner_probe_last_tenth": [min(pr_last), max(pr_last)],
                "cycles_per_solve_last": float(np.mean(cyc[-min(len(cyc), 5000):])) if len(cyc) else None,
                "vortices": sorted(k for k in vortex_census(self.cav.psi()) if k != "primary"),
                "monitors": h}


def run_cases(cases, t_end, every, max_seconds):
    t0 = time.perf_counter()
    while True:
        live = [c for c in cases if c.steps * c.dt < t_end - 1e-12 and c.steady_at is None and c.error is None]
        if not live or time.perf_counter() - t0 > max_seconds:
            break
        for c in live:
            n = min(every, int(round((t_end - c.steps * c.dt) / c.dt)))
            if n > 0:
                try:
                    rec = c.advance(n)
                except Exception as e:  # a diverged case stops; the others go on
                    c.error = f"{type(e).__name__} at t = {c.steps * c.dt:g}: {e}"
                    print(json.dumps({"case": c.name, "error": c.error}), file=sys.stderr, flush=True)
                    continue
                if len(c.hist) % 20 == 0:
                    print(json.dumps({"case": c.name, **rec}), file=sys.stderr, flush=True)


def floor(args):
    from paper_0809_3098_gb300 import lc

    MIXED = lc.LC_PREC_MIXED
    base = Case("rhs64=1 (from rest)", args.N, args.Re, args.dt, precision=MIXED, rhs64=1)
    run_cases([base], args.t_branch, args.every, args.max_seconds)
    psi, omega = base.cav.psi(), base.cav.omega()
    out = {"branch_t": sig(base.steps * base.dt, 6), "phase1": base.summary()}
    base.cav.close()
    branches = [Case("rhs64=1", args.N, args.Re, args.dt, precision=MIXED, rhs64=1),
                Case("rhs64=0", args.N, args.Re, args.dt, precision=MIXED, rhs64=0)]
    for b in branches:
        b.cav.set_state(psi, omega)
        b.steps = int(round(args.t_branch / b.dt))
    run_cases(branches, args.t_end, args.every, args.max_seconds)
    out["branches"] = [b.summary() for b in branches]
    return out


def coarse(args):
    from paper_0809_3098_gb300 import lc

    MIXED = lc.LC_PREC_MIXED
    N, Re = args.N, args.Re
    cases = [Case(f"multigrid to 1e-10, mixed, dt={dt:g}", N, Re, dt, precision=MIXED) for dt in args.mg_dts]
    if args.fp64:
        cases.append(Case(f"multigrid to 1e-10, FP64, dt={args.dt:g}", N, Re, args.dt))
    for beta, sweeps in args.sor:
        cases.append(Case(f"SOR beta={beta} sweeps/stage={sweeps}, dt={args.dt:g}", N, Re, args.dt, tol=1e30,
                          solver=1, beta=beta, sor_sweeps=sweeps))
    run_cases(cases, args.t_end, args.every, args.max_seconds)
    return {"cases": [c.summary() for c in cases]}


def paper(args):
    from paper_0809_3098_gb300 import lc

    cases = [Case(f"Re {Re:g}", args.N, Re, args.dt, precision=lc.LC_PREC_MIXED) for Re in args.Res]
    run_cases(cases, args.t_end, args.every, args.max_seconds)
    return {"cases": [c.summary() for c in cases]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["floor", "coarse", "paper"])
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--Re", type=float, default=None)
    ap.add_argument("--Res", type=float, nargs="+", default=[10000.0, 20000.0, 30000.0])
    ap.add_argument("--dt", type=float, default=0.001)
    ap.add_argument("--t-branch", type=float, default=150.0)
    ap.add_argument("--t-end", type=float, default=None)
    ap.add_argument("--every", type=int, default=None)
    ap.add_argument("--sor", type=lambda s: tuple(float(x) if "." in x else int(x) for x in s.split(":")),
                    nargs="*", default=[(0.5, 1), (0.5, 10)], help="beta:sweeps per stage")
    ap.add_argument("--fp64", action="store_true", help="coarse: add the FP64 multigrid case")
    ap.add_argument("--mg-dts", type=float, nargs="*", default=[0.001, 0.0005],
                    help="coarse: time steps of the multigrid cases")
    ap.add_argument("--max-seconds", type=float, default=1e9)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    defaults = {"floor": (1024, 5000.0, 270.0, 2000), "coarse": (224, 10000.0, 200.0, 250),
                "paper": (1024, None, 100.0, 2000)}[args.mode]
    args.N = args.N or defaults[0]
    args.Re = args.Re or defaults[1]
    args.t_end = args.t_end or defaults[2]
    args.every = args.every or defaults[3]
    import torch

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    out = {"command": "python -m tests.studies.long_runs " + " ".join(sys.argv[1:]), "mode": args.mode}
    out.update({"floor": floor, "coarse": coarse, "paper": paper}[args.mode](args))
    out["seconds"] = round(time.perf_counter() - t0, 1)
    text = json.dumps(out, separators=(",", ":"))
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
