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

and the driven-particle benchmark of Sec. 3.2 (one bead in a box periodic in
x and y, H = 10 d, pushed by a constant force F_0 against a uniform counter
force on the fluid):

  internal-flow  eps_v / V_0^2 against r_eta (r_xi = 0.01, Fig. 3d), against
              r_xi (r_eta = 100, Fig. 3e) and against Re_p; with each point the
              drag F_0 / (eta V_0) against Hasimoto's periodic array of rigid
              discs and the disc radius that reproduces it

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


# One rigid tumbling case (Sec. 4.2: K = 3.3, C = 0.2, Re_ps = 0.25, N = 10
# beads of a = 2, r_eta = 100, r_xi = 0.125, L_x = 25 d) and variants that
# each change one reading or numerical choice, to find what sets the period:
# (label, overrides of tumbling_case's arguments, overrides of the config).
READINGS = [
    ("base", {}, {}),
    ("r_eta 50", dict(r_eta=50.0), {}),
    ("r_eta 300", dict(r_eta=300.0), {}),
    ("r_eta 1000", dict(r_eta=1000.0), {}),
    ("K 33", dict(K=33.0), {}),
    ("K 330", dict(K=330.0), {}),
    ("k_s x10", {}, dict(k_s="x10")),
    ("phi_cut 4", {}, dict(phi_cut=4.0)),
    ("Re_ps 0.1", dict(Re_ps=0.1), {}),
    ("C 0.1", dict(C=0.1, U=0.04), {}),
    ("L_x 50 d", dict(lx_over_d=50.0), {}),
    ("a 4", dict(a=4.0, U=0.04), {}),
    ("a 4, r_xi 0.0625", dict(a=4.0, U=0.04, r_xi=0.0625), {}),
    ("a 4, r_xi 0.25", dict(a=4.0, U=0.04, r_xi=0.25), {}),
    ("LL rates", {}, dict(collision=1)),
    ("N 2", dict(N=2), {}),
    ("N 2, r_eta 1000", dict(N=2, r_eta=1000.0), {}),
]


# The interface-width series of the rigid case: beads of a = 8 cells (so that
# thin interfaces stay resolved), r_xi = xi / d from 0.125 down to 1/64, and
# the viscosity ratio at the thinnest interfaces.
INTERFACE = [
    ("a 8, r_xi 0.125", dict(a=8.0, U=0.04), {}),
    ("a 8, r_xi 0.0625", dict(a=8.0, U=0.04, r_xi=0.0625), {}),
    ("a 8, r_xi 0.03125", dict(a=8.0, U=0.04, r_xi=0.03125), {}),
    ("a 8, r_xi 0.015625", dict(a=8.0, U=0.04, r_xi=0.015625), {}),
    ("a 8, r_xi 0.03125, r_eta 20", dict(a=8.0, U=0.04, r_xi=0.03125, r_eta=20.0), {}),
    ("a 8, r_xi 0.03125, r_eta 500", dict(a=8.0, U=0.04, r_xi=0.03125, r_eta=500.0), {}),
]


def readings(precision: int = 1, variants=READINGS) -> dict:
    """gamma_dot T (180-degree turn) and the aspect ratio r_e fitted to
    omega(theta) by Eq. 19 for each variant of the rigid tumbling case, beside
    Jeffery's pi (r + 1/r) for the geometric r_c = 1/N and for r_e."""
    cases = []
    for label, kw, over in variants:
        base = dict(K=RIGID, C=0.2, Re_ps=0.25)
        base.update(kw)
        K, C, Re_ps = base.pop("K"), base.pop("C"), base.pop("Re_ps")
        cfg, g = tb.tumbling_case(K, C, Re_ps, **base)
        for k, v in over.items():
            if v == "x10":
                d = 2.0 * cfg["a"]
                cfg[k] = 10 * 0.25 * math.pi * cfg["a"] ** 2 * d * d
            else:
                cfg[k] = v
        cases.append((label, cfg, g, 1.0 / cfg["n_beads"]))
    g_min = min(g / (1.0 / r + r) for _, _, g, r in cases)
    res = tb.measure_periods([c for _, c, _, _ in cases], int(2.2 * math.pi / g_min),
                             sample_every=100, precision=precision)
    rows = []
    for (label, cfg, g, r_c), r in zip(cases, res):
        t, th, e2e = r.track.arrays()
        row = dict(variant=label, nx=cfg["nx"], ny=cfg["ny"], gamma_dot=g, gT=r.T * g,
                   gT_jeffery_geometric=tb.jeffery_half_period(r_c, 1.0),
                   min_e2e=float(e2e.min()) if len(e2e) else float("nan"))
        if math.isfinite(r.T) and len(t) > 10:
            keep = t > 0.3 * r.T
            r_fit, rms = tb.jeffery_fit(t[keep], th[keep], g)
            row.update(r_fit=r_fit, fit_rms=rms, gT_jeffery_fitted=tb.jeffery_half_period(r_fit, 1.0))
        rows.append(row)
    return dict(study="readings", rows=rows)


def sensitivity(checkpoints=(2000, 10000, 50000, 100000, 200000), seed: int = 7) -> dict:
    """How much the FP64 trajectory of the 1024 x 256 flexible-fiber case
    (K = 3.3e-5, Re = 10) moves when its initial populations are perturbed
    by one ulp, by the FP32 unit roundoff (6e-8 of each deviation f - w, random
    sign) and by the FP16 one (4.9e-4), against the FP32- and FP16-storage runs
    of the same case: velocity relative L2 and largest bead displacement
    against the unperturbed FP64 run at each checkpoint.  A trajectory that
    amplified perturbations would carry the perturbed runs as far as the
    reduced-precision ones; a stable one keeps them near their start."""
    from . import fpd, workloads as wl
    base = wl.single_fiber_medium()
    rng = np.random.default_rng(seed)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]

    def make(prec, pert=None):
        s = fpd.Simulation(dict(base, precision=prec))
        if pert is not None:
            f = s.populations()
            if pert == "ulp":
                f2 = np.nextafter(f, np.inf)
            else:
                f2 = f + (f - w) * pert * rng.choice([-1.0, 1.0], size=f.shape)
            s.set_populations(f2)
        return s

    sims = {"ref": make(0), "ulp": make(0, "ulp"), "fp32_roundoff": make(0, 6e-8),
            "fp16_roundoff": make(0, 4.9e-4), "fp32_storage": make(1), "fp16_storage": make(2)}
    rows = []
    done = 0
    for c in checkpoints:
        for sim in sims.values():
            sim.step(c - done)
        done = c
        ux, uy, _ = sims["ref"].fields()
        ref_u, ref_R = np.stack([ux, uy]), sims["ref"].beads()[0]
        row = dict(steps=c)
        for k, sim in sims.items():
            if k == "ref":
                continue
            a, b, _ = sim.fields()
            R = sim.beads()[0]
            row[k] = dict(u=float(np.linalg.norm(np.stack([a, b]) - ref_u) / np.linalg.norm(ref_u)),
                          dR=float(np.abs(R - ref_R).max()))
        rows.append(row)
    for sim in sims.values():
        sim.close()
    return dict(study="sensitivity", case=base["name"], rows=rows)


def hasimoto_drag(a: float, L: float) -> float:
    """F / (eta V) of a square array (period L) of rigid discs of radius a in
    Stokes flow (Hasimoto 1959), to third order in the area fraction c."""
    c = math.pi * a * a / (L * L)
    return 4 * math.pi / (-0.5 * math.log(c) - 0.738 + c - 0.887 * c * c + 2.039 * c ** 3)


def hasimoto_radius(k: float, L: float) -> float:
    """Disc radius whose periodic-array drag F / (eta V) equals k (bisection)."""
    lo, hi = 1e-3 * L, 0.45 * L
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if hasimoto_drag(mid, L) < k:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def driven_case(a: float, r_eta: float, r_xi: float, Re_p: float, h_over_d: float = 10.0,
                nu: float = 1.0 / 6.0) -> dict:
    """One bead of radius a in a periodic box of side h_over_d * d, driven
    along x by F_0 chosen from Hasimoto's drag for a target Re_p = V_0 d / nu;
    the fluid carries the counter force -F_0 / L^2 (Sec. 3.2)."""
    d = 2.0 * a
    L = int(round(h_over_d * d))
    V0 = Re_p * nu / d
    F0 = hasimoto_drag(a, L) * nu * V0
    return dict(nx=L, ny=L, u_bottom=0.0, u_top=0.0, nu_f=nu, re=1.0, visc_ratio=r_eta, xi=r_xi * d, a=a,
                n_beads=1, n_fibers=1, k_s=-1.0, k_b=0.0, stiffness_K=0.0, k_ev=-1.0, phi_cut=8.0,
                gx=-F0 / (L * L), gy=0.0, collision=0, s_e=1.64, s_eps=1.54, s_q=1.9, init_couette=0,
                periodic_y=1, bead_fx=F0, bead_fy=0.0, centres=[[L / 2.0, L / 2.0]], theta0=[0.0])


INTERNAL_FLOW = (
    [("r_eta", r, 0.01, 0.1) for r in (1.0, 2.0, 5.0, 10.0, 20.0, 50.0, 100.0, 200.0)]
    + [("r_xi", 100.0, x, 0.1) for x in (0.01, 0.03, 0.0625, 0.125, 0.25)]
    + [("Re_p", 100.0, 0.0625, r) for r in (0.1, 1.0, 3.0)]
)


def internal_flow(a: float = 8.0, precision: int = 1, points=INTERNAL_FLOW, viscous_times: float = 3.0) -> dict:
    from . import fpd
    cfgs = [driven_case(a, r_eta, r_xi, Re_p) for _, r_eta, r_xi, Re_p in points]
    nu, L, d = cfgs[0]["nu_f"], cfgs[0]["nx"], 2.0 * a
    steps = int(viscous_times * L * L / nu)
    cells = sum(c["nx"] * c["ny"] for c in cfgs)
    es = {0: 8, 1: 4, 2: 2}[precision]
    b = fpd.Batch(precision, len(cfgs), 18 * es * (cells + 64 * L * len(cfgs)) + 4096 * len(cfgs), len(cfgs))
    slots = [b.add(dict(c, precision=precision), steps) for c in cfgs]
    b.run(int(0.9 * steps))
    V_early = [b.beads(s)[1][0, 0] for s in slots]
    while b.run(steps):
        pass
    rows = []
    for (group, r_eta, r_xi, Re_t), c, s, ve in zip(points, cfgs, slots, V_early):
        V = b.beads(s)[1][0, 0]
        eps = float(b.internal_flow(s)[0])
        k = c["bead_fx"] / (nu * V)
        rows.append(dict(group=group, r_eta=r_eta, r_xi=r_xi, Re_p=V * d / nu, eps_rel=eps / V ** 2,
                         drag=k, drag_over_hasimoto=k / hasimoto_drag(a, L),
                         a_eff_over_a=hasimoto_radius(k, L) / a, V_drift=abs(V / ve - 1)))
    b.close()
    return dict(study="internal-flow", a=a, L=L, nu=nu, steps=steps, rows=rows)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["resolution", "internal-flow", "readings", "interface", "sensitivity"]
                    + sorted(SWEEPS))
    ap.add_argument("--a", type=float, default=2.0, help="bead radius in lattice units")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1, 2])
    args = ap.parse_args(argv)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("the studies run on the CUDA library: no CUDA device")
    from . import build
    build.build()
    if args.study == "resolution":
        out = resolution(precision=args.precision)
    elif args.study == "readings":
        out = readings(precision=args.precision)
    elif args.study == "interface":
        out = readings(precision=args.precision, variants=INTERFACE)
    elif args.study == "sensitivity":
        out = sensitivity()
    elif args.study == "internal-flow":
        out = internal_flow(a=args.a if args.a != 2.0 else 8.0, precision=args.precision)
    else:
        out = sweep(args.study, a=args.a, precision=args.precision)
    print(json.dumps(out, indent=1, default=float))


if __name__ == "__main__":
    main()
