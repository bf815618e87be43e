"""Long-time study: several lid-driven cavities advanced together by the
batched mixed-precision engine towards steady state, with the steady-state
monitors of Eqs. (26)-(27) every `--every` steps and a census of the corner
vortices at the end (Cardoso & Bicudo, arXiv:0809.3098, Sec. 3.2 and the
vortex discussion of Sec. 4).

Each cavity is "N:Re" (N intervals per side).  dt is the paper's 0.001 unless
--dt says otherwise (0 = the rule 0.25 min(h, Re h^2 / 4)).  A cavity counts
as steady once RES_psi < 1e-12 and RES_omega < 1e-10 (the paper's thresholds
for Re <= 20000; 1e-10 and 1e-8 above).  The monitors are computed on the
host from the states before and after one step, with the oracle's monitor
formula.

Vortex census: the connected regions of psi > 0 and psi < 0 over interior
nodes (4-connectivity).  The largest psi < 0 region is the primary vortex;
every other region is named by the corner quadrant holding its extremum
(BL, BR, TL, TR) and numbered by size within that corner, which is the
naming of the paper's schematic (TL1, BL1, BL2, ...).

    python -m tests.studies.steady_study --cavities 224:5000 224:10000 320:15000 \
        --t-end 300 > steady.json
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def vortex_census(psi: np.ndarray, min_area: int = 2, min_abs: float = 1e-13):
    from scipy import ndimage

    N = psi.shape[0] - 1
    inner = psi[1:-1, 1:-1]
    regions = []
    for sign in (1, -1):
        lab, n = ndimage.label(sign * inner > 0)
        for k in range(1, n + 1):
            idx = lab == k
            area = int(idx.sum())
            vals = inner[idx]
            ext = float(vals.max() if sign > 0 else vals.min())
            if area < min_area or abs(ext) < min_abs:
                continue
            jj, ii = np.argwhere(idx & (inner == ext))[0]
            regions.append({"sign": sign, "area": area / (N - 1) ** 2, "psi_extremum": ext,
                            "x": (ii + 1) / N, "y": (jj + 1) / N})
    neg = [r for r in regions if r["sign"] < 0]
    primary = max(neg, key=lambda r: r["area"]) if neg else None
    named = {}
    for r in regions:
        if r is primary:
            continue
        corner = ("T" if r["y"] >= 0.5 else "B") + ("R" if r["x"] >= 0.5 else "L")
        named.setdefault(corner, []).append(r)
    out = {"primary": primary}
    for corner, rs in named.items():
        rs.sort(key=lambda r: -r["area"])
        for k, r in enumerate(rs, 1):
            out[f"{corner}{k}"] = r
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cavities", nargs="+", default=["224:5000", "224:10000", "320:10000", "320:15000"])
    ap.add_argument("--dt", type=float, default=0.001)
    ap.add_argument("--t-end", type=float, default=300.0)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--max-seconds", type=float, default=1e9)
    args = ap.parse_args()
    import torch

    import oracle
    from paper_0809_3098_gb300 import lc

    torch.cuda.set_device(0)
    Ns = [int(c.split(":")[0]) for c in args.cavities]
    Res = [float(c.split(":")[1]) for c in args.cavities]
    dts = [args.dt] * len(Ns)
    b = lc.Batch(Ns, Res, dts)
    nu = b.autotune_schedule(steps=2)
    dt_used = [b.info(c)["dt"] for c in range(len(Ns))]
    thresholds = [(1e-12, 1e-10) if Re <= 20000 else (1e-10, 1e-8) for Re in Res]
    hist = [[] for _ in Ns]
    steady_at = [None] * len(Ns)
    steps_total = int(round(args.t_end / min(dt_used)))
    t0 = time.perf_counter()
    done = 0
    while done < steps_total:
        n = min(args.every - 1, steps_total - done - 1)
        if n > 0:
            b.step(n)
        before = [(b.psi(c), b.omega(c)) for c in range(len(Ns))]
        b.step(1)
        done += n + 1
        for c in range(len(Ns)):
            p1, w1 = b.psi(c), b.omega(c)
            m = oracle.monitors(Ns[c], dt_used[c], before[c][0], p1, before[c][1], w1)
            hist[c].append({"step": done, "t": done * dt_used[c], "max_domega_dt": float(m[0]),
                            "RES_psi": float(m[1]), "RES_omega": float(m[2]),
                            "psi_min": float(p1.min())})
            if steady_at[c] is None and m[1] < thresholds[c][0] and m[2] < thresholds[c][1]:
                steady_at[c] = done
        if all(s is not None for s in steady_at) or time.perf_counter() - t0 > args.max_seconds:
            break
    b.synchronize()
    seconds = time.perf_counter() - t0
    out = {"dt": dt_used, "steps": done, "seconds": seconds, "schedule": nu, "cavities": []}
    for c in range(len(Ns)):
        h = hist[c]
        tail = [r["max_domega_dt"] for r in h[-10:]]
        out["cavities"].append({
            "N": Ns[c], "Re": Res[c], "dt": dt_used[c], "t_end": done * dt_used[c],
            "steady_at_step": steady_at[c], "thresholds": thresholds[c],
            "monitors": h,
            "tail_max_domega_dt": {"min": min(tail), "max": max(tail), "last": tail[-1]},
            "vortices": vortex_census(b.psi(c)),
            "vcycles_per_solve": float(b.cycle_log(c)[-5000:].mean()),
        })
        print(json.dumps({k: v for k, v in out["cavities"][-1].items() if k != "monitors"}), file=sys.stderr,
              flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
