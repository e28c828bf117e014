"""Seeded synthetic inputs shaped like the paper's Couette-fiber runs.

This module only draws and lists raw problem parameters (lattice size, wall
speeds, Re, stiffness parameter K, bead count/radius, fiber centres and seeded
angles).  It holds none of the method's arithmetic: every derived quantity
(viscosity from Re, bending constant from K, relaxation rates, bead positions
from centre and angle) is computed independently by the CUDA library and by
the CPU oracle.  Both consume the dicts returned here.

Geometry of every case follows Sec. 4.1 of the paper: a single-phase fluid
between walls at y = 0 and y = H moving at -U and +U, periodic in x, fibers of
N beads of radius a centred between the walls.  "re" is gamma_dot l_c^2 / nu_f
(the paper's Re_ps is re / 4); "stiffness_K" is K of Eq. 18.
"""
from __future__ import annotations

import math

import numpy as np

PRECISION_F64 = 0
PRECISION_F32 = 1
PRECISION_F16 = 2

_BASE = dict(
    u_bottom=-0.01, u_top=0.01, nu_f=-1.0, visc_ratio=50.0, k_s=-1.0, k_b=0.0,
    k_ev=-1.0, phi_cut=8.0, gx=0.0, gy=0.0, collision=0, s_e=1.64, s_eps=1.54,
    s_q=1.9, init_couette=1,
)


def _angle(rng: np.random.Generator, lo_deg=30.0, hi_deg=60.0) -> float:
    return math.radians(float(rng.uniform(lo_deg, hi_deg)))


def single_fiber_small(seed: int = 1) -> dict:
    """80 x 40 lattice, walls -/+0.01, one 8-bead fiber (a = 2, spacing 2a),
    centred, seeded angle in [30, 60] deg, r_eta = 50, xi = 1, stiff bending
    (K = 3.3), Re = 1; run for 10 000 steps in FP64."""
    rng = np.random.default_rng(seed)
    return dict(_BASE, nx=80, ny=40, re=1.0, xi=1.0, a=2.0, n_beads=8, n_fibers=1,
                stiffness_K=3.3, centres=[[40.0, 20.0]], theta0=[_angle(rng)],
                precision=PRECISION_F64, steps=10_000,
                name="single_fiber_80x40_N8_fp64")


def single_fiber_medium(seed: int = 2, precision: int = PRECISION_F32) -> dict:
    """1024 x 256 lattice, one 20-bead fiber (a = 4), r_eta = 50, fairly
    flexible (K = 3.3e-5), Re = 10, seeded angle; 200 000 steps."""
    rng = np.random.default_rng(seed)
    return dict(_BASE, nx=1024, ny=256, re=10.0, xi=1.0, a=4.0, n_beads=20, n_fibers=1,
                stiffness_K=3.3e-5, centres=[[512.0, 128.0]], theta0=[_angle(rng)],
                precision=precision, steps=200_000,
                name="single_fiber_1024x256_N20")


def two_fiber_large(seed: int = 3, precision: int = PRECISION_F32) -> dict:
    """4096 x 1024 lattice, two 20-bead fibers (a = 4) at x = Lx/4 and 3Lx/4,
    r_eta = 50, K = 0.33, Re = 5, seeded angles."""
    rng = np.random.default_rng(seed)
    return dict(_BASE, nx=4096, ny=1024, re=5.0, xi=1.0, a=4.0, n_beads=20, n_fibers=2,
                stiffness_K=0.33, centres=[[1024.0, 512.0], [3072.0, 512.0]],
                theta0=[_angle(rng), _angle(rng)], precision=precision, steps=20_000,
                name="two_fiber_4096x1024_N20")


def sweep_instance(rng: np.random.Generator, precision: int = PRECISION_F32) -> dict:
    """One point of the confinement / Re / stiffness sweep: H ~ U{32..256},
    width 2H, C ~ U[0.2, 0.8], a ~ U[2, 4], N = clamp(round(C H / 2a), 3, 30),
    Re ~ U[1, 10], K log-uniform over [3.3e-3, 3.3], xi = a / 4, seeded angle.
    The wall speed is 0.01 unless the fluid relaxation time would drop below
    0.51, in which case it is raised just enough (capped at 0.05)."""
    H = int(rng.integers(32, 257))
    C = float(rng.uniform(0.2, 0.8))
    a = float(rng.uniform(2.0, 4.0))
    N = int(min(30, max(3, round(C * H / (2.0 * a)))))
    re = float(rng.uniform(1.0, 10.0))
    K = float(10.0 ** rng.uniform(math.log10(3.3e-3), math.log10(3.3)))
    lc = 2.0 * a * N
    # nu_f = (2U/H) lc^2 / re must keep 3 nu_f + 1/2 >= 0.51
    U = 0.01
    nu_min = 0.01 / 3.0
    U_need = nu_min * H * re / (2.0 * lc * lc)
    if U_need > U:
        U = min(0.05, U_need * 1.0001)
    return dict(_BASE, nx=2 * H, ny=H, u_bottom=-U, u_top=U, re=re, xi=a / 4.0, a=a,
                n_beads=N, n_fibers=1, stiffness_K=K, centres=[[float(H), H / 2.0]],
                theta0=[_angle(rng)], precision=precision)


def batched_sweep(n: int = 512, seed: int = 4, precision: int = PRECISION_F32) -> list[dict]:
    """The batched sweep: n independent instances drawn by ``sweep_instance``."""
    rng = np.random.default_rng(seed)
    return [sweep_instance(rng, precision) for _ in range(n)]


def serving_requests(n: int, rate_per_s: float, seed: int = 5, steps_lo: int = 50_000,
                     steps_hi: int = 500_000, precision: int = PRECISION_F32) -> list[dict]:
    """Poisson arrivals (seeded) of sweep instances, each with a step count
    drawn uniformly in [steps_lo, steps_hi]; 'arrival_s' is the arrival time."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        inst = sweep_instance(rng, precision)
        inst["steps"] = int(rng.integers(steps_lo, steps_hi + 1))
        inst["arrival_s"] = t
        out.append(inst)
    return out


def couette_only(nx: int, ny: int, u: float = 0.01, nu: float = 0.1, init_couette: int = 1,
                 precision: int = PRECISION_F64) -> dict:
    """Plain Couette cell without fibers."""
    return dict(_BASE, nx=nx, ny=ny, u_bottom=-u, u_top=u, nu_f=nu, re=1.0, xi=1.0, a=2.0,
                n_beads=0, n_fibers=0, stiffness_K=0.0, centres=[[0.0, 0.0]], theta0=[0.0],
                init_couette=init_couette, precision=precision)


def random_fiber(rng: np.random.Generator, nx: int, ny: int, n_beads: int, a: float, xi: float,
                 n_fibers: int = 1, precision: int = PRECISION_F64, **over) -> dict:
    """A small randomised case for parity tests: random wall speeds, Re,
    stiffness, centre and angle; any key may be overridden."""
    U = float(rng.uniform(0.005, 0.02))
    cen = []
    for f in range(n_fibers):
        cen.append([float((f + 0.5) * nx / n_fibers + rng.uniform(-1, 1)),
                    float(ny / 2 + rng.uniform(-1, 1))])
    d = dict(_BASE, nx=nx, ny=ny, u_bottom=-U, u_top=U, re=float(rng.uniform(1, 10)), xi=xi,
             a=a, n_beads=n_beads, n_fibers=n_fibers,
             stiffness_K=float(10 ** rng.uniform(-3, 0.5)), centres=cen,
             theta0=[float(rng.uniform(0, math.pi)) for _ in range(n_fibers)],
             precision=precision)
    d.update(over)
    return d
