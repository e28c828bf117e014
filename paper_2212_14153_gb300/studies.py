"""Tumbling-period studies of Sec. 4 on the batched engine.

Each study is a list of tumbling configurations (one fiber of N = 10 beads,
r_c = 1/N, between walls at -U and +U) advanced together by the CUDA
library; the period of each is measured by ``tumbling.measure_periods`` and
the divergence law gamma_dot T ~ (x_cr - x)^-beta is fitted where the period
grows toward a critical Re_ps or confinement C:

  resolution  rigid fiber (K = 3.3), C = 0.2, Re_ps = 0.25, bead radius
              a = 2 .. 8 cells at fixed r_xi = xi / d: the period against
              Jeffery's (Eq. 19) with the geometric and the fitted aspect ratio
  rigid-re    rigid fiber, C = 0.2, Re_ps swept (Fig. 5b: beta = 1/2)
  rigid-re-n2 the same for a two-bead fiber, r_c = 1/2 (Fig. 5b, open diamonds)
  rigid-c     rigid fiber, Re_ps = 1.5, C swept (Fig. 5c: beta = 1/2)
  flex-re     fairly flexible fiber (K = 3.3e-5), C = 0.5, Re_ps swept (Fig. 8a: beta = 0.3)
  flex-c      fairly flexible fiber, Re_ps = 1.5, C swept (Fig. 8b: beta = 0.6)

Run: python -m paper_2212_14153_gb300.studies <study> [--a A] [--precision P]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import tumbling as tb

RIGID, FLEXIBLE = 3.3, 3.3e-5

# (stiffness K, swept variable, values, the other variable's value, the
# paper's beta, smallest x of the fitted range: the C-law of Sec. 4.2 holds
# for C >= 0.5, below which T barely depends on C)
SWEEPS = {
    "rigid-re": (RIGID, "Re_ps", [0.25, 0.5, 1.0, 1.5, 1.75, 2.0, 2.25, 2.5, 3.0, 6.0], 0.2, 0.5, 0.0),
    "rigid-re-n2": (RIGID, "Re_ps", [0.5, 1.0, 2.0, 4.0, 6.0, 7.0, 8.0, 8.5, 9.0, 10.0, 12.0], 0.2, 0.5, 0.0),
    "rigid-c": (RIGID, "C", [0.1, 0.2, 0.3, 0.4, 0.5, 0.55, 0.6, 0.65, 0.675, 0.7, 0.8], 1.5, 0.5, 0.5),
    "flex-re": (FLEXIBLE, "Re_ps", [0.5, 1.0, 1.5, 2.0, 2.25, 2.5, 2.75, 3.0, 4.0, 6.0], 0.5, 0.3, 0.0),
    "flex-c": (FLEXIBLE, "C", [0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.75, 0.8, 0.85, 0.9], 1.5, 0.6, 0.0),
}


def _budget(g: float, turns: float = 6.0) -> int:
    """Steps for `turns` Jeffery half periods of the geometric r_c = 0.1."""
    return int(turns * tb.jeffery_half_period(0.1, g))


def resolution(radii=(2.0, 3.0, 4.0, 6.0, 8.0), precision: int = 1, Re_ps: float = 0.25) -> dict:
    cases = [tb.tumbling_case(RIGID, 0.2, Re_ps, a=a) for a in radii]
    gs = [g for _, g in cases]
    res = tb.measure_periods([c for c, _ in cases], _budget(min(gs), 3.0),
                             sample_every=max(50, int(tb.jeffery_half_period(0.1, max(gs)) / 600)),
                             precision=precision)
    rows = []
    for a, (cfg, g), r in zip(radii, cases, res):
        t, th, _ = r.track.arrays()
        keep = t > 0.3 * (r.T if math.isfinite(r.T) else t[-1])
        r_fit, rms = tb.jeffery_fit(t[keep], th[keep], g)
        rows.append(dict(a=a, nx=cfg["nx"], ny=cfg["ny"], gT=r.T * g, r_fit=r_fit, fit_rms=rms,
                         gT_jeffery_geometric=tb.jeffery_half_period(0.1, 1.0),
                         gT_jeffery_fitted=tb.jeffery_half_period(r_fit, 1.0)))
    return dict(study="resolution", Re_ps=Re_ps, C=0.2, rows=rows)


def sweep(name: str, a: float = 2.0, precision: int = 1, values=None) -> dict:
    K, var, vals, other, beta, x_min = SWEEPS[name]
    values = vals if values is None else values
    N = 2 if name.endswith("-n2") else 10
    cases = []
    for v in values:
        Re_ps, C = (v, other) if var == "Re_ps" else (other, v)
        cases.append(tb.tumbling_case(K, C, Re_ps, N=N, a=a))
    gs = [g for _, g in cases]
    r_c = 1.0 / N
    res = tb.measure_periods([c for c, _ in cases], _budget(min(gs)),
                             sample_every=max(50, int(tb.jeffery_half_period(r_c, max(gs)) / 400)),
                             precision=precision)
    rows = [dict(x=v, nx=c["nx"], ny=c["ny"], gT=r.T * g, stuck_deg=r.stuck_deg)
            for v, (c, g), r in zip(values, cases, res)]
    fin = [r for r in rows if math.isfinite(r["gT"]) and r["x"] >= x_min]
    x = np.array([r["x"] for r in fin])
    T = np.array([r["gT"] for r in fin])
    stuck = [r["x"] for r in rows if not math.isfinite(r["gT"])]
    out = dict(study=name, K=K, N=N, variable=var, other=other, a=a, fit_range=[x_min, None], rows=rows,
               bracket=[float(x.max()) if len(x) else None, min(stuck) if stuck else None])
    if len(x) >= 3:
        x_cr, T0, rms = tb.critical_fit(x, T, beta)
        out["fit_paper_beta"] = dict(beta=beta, x_cr=x_cr, gT0=T0, rms=rms)
        # the same law through the three tumbling points nearest the divergence
        x_cr3, _, rms3 = tb.critical_fit(x[-3:], T[-3:], beta)
        out["fit_near_critical"] = dict(beta=beta, x_cr=x_cr3, rms=rms3, points=x[-3:].tolist())
        try:
            x_cr, T0, b, rms = tb.critical_fit_beta(x, T)
            out["fit_free_beta"] = dict(beta=b, x_cr=x_cr, gT0=T0, rms=rms)
        except ValueError:
            pass
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["resolution"] + sorted(SWEEPS))
    ap.add_argument("--a", type=float, default=2.0, help="bead radius in lattice units")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1, 2])
    args = ap.parse_args(argv)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("the studies run on the CUDA library: no CUDA device")
    from . import build
    build.build()
    out = resolution(precision=args.precision) if args.study == "resolution" else \
        sweep(args.study, a=args.a, precision=args.precision)
    print(json.dumps(out, indent=1, default=float))


if __name__ == "__main__":
    main()
