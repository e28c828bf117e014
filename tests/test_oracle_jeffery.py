"""Whole coupled step of the oracle against Jeffery's orbit (Sec. 4.2, Eq. 19).

A stiff fiber (K = 3.3) at weak confinement (C = 0.2) and small Reynolds
number (Re = 1, i.e. Re_ps = 0.25) must tumble clockwise with an angular
velocity of Jeffery's form omega = (g/2)[A cos 2 theta - 1],
A = (1 - r_e^2)/(1 + r_e^2).  As in the paper, r_e is obtained by a least-
squares fit of omega(theta); the measured full-revolution period must then
agree within 5% with 2 pi (r_e + 1/r_e) / gamma_dot (two 180-degree turns, the
paper's period T being one of them).  The paper reports the fitted r_e to be
larger than the geometric d / l_c (0.132 vs 0.1); at the coarse resolution used
here (bead diameter 4 cells) the ratio is larger still, and the test bounds it
loosely to [1, 2.2] x d / l_c.
"""
import math
import os

import numpy as np
import pytest

import oracle


def _run_half_turn(N=6, a=2.0, xi=0.5, C=0.2, U=0.05, Re=1.0, Lx=80):
    lc = N * 2 * a
    H = int(round(lc / C))
    cfg = dict(nx=Lx, ny=H, u_bottom=-U, u_top=U, re=Re, visc_ratio=50.0, xi=xi, a=a,
               n_beads=N, n_fibers=1, stiffness_K=3.3, centres=[[Lx / 2, H / 2]],
               theta0=[math.pi / 2], threads=min(8, os.cpu_count() or 1))
    s = oracle.Sim(cfg)
    gd = s.derived()["gamma_dot"]
    prev = math.pi / 2
    ts, ths = [0.0], [prev]
    unwrapped = prev
    while unwrapped > -math.pi / 2 - 0.05:
        s.step(100)
        th = oracle.fiber_angle(s.beads()[0], N)
        d = th - prev
        d -= math.pi * round(d / math.pi)      # fiber is head-tail symmetric
        unwrapped += d
        prev = th
        ts.append(float(s.nstep))
        ths.append(unwrapped)
        assert s.nstep < 200_000
    return np.array(ts), np.array(ths), gd, N


@pytest.mark.slow
def test_stiff_fiber_follows_jeffery_orbit():
    ts, ths, gd, N = _run_half_turn()
    # time of one 180-degree turn, from theta = 90 deg to -90 deg
    i = int(np.argmax(ths <= -math.pi / 2))
    t180 = ts[i - 1] + (-math.pi / 2 - ths[i - 1]) / (ths[i] - ths[i - 1]) * (ts[i] - ts[i - 1])
    omega = np.gradient(ths, ts)
    keep = ts > 2000                                   # skip the start-up transient
    assert np.all(omega[keep] < 0)                      # clockwise tumbling
    c2 = (gd / 2) * np.cos(2 * ths[keep])
    A = float(np.sum((omega[keep] + gd / 2) * c2) / np.sum(c2 * c2))
    resid = omega[keep] - (gd / 2) * (A * np.cos(2 * ths[keep]) - 1)
    assert np.sqrt(np.mean(resid ** 2)) < 0.05 * gd     # Eq. 19 shape holds
    r_e = math.sqrt((1 - A) / (1 + A))
    assert 1.0 / N <= r_e <= 2.2 / N
    T_jeffery = 2 * math.pi * (r_e + 1 / r_e) / gd
    assert abs(2 * t180 / T_jeffery - 1) < 0.05
