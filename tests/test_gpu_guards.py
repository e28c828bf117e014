"""Device-side guards and diagnostics against the oracle and closed forms.

- fpd_diag's mass and momentum against the oracle's totals (FP64, 1e-12).
- Eq. 5 on the GPU: the bead velocity in a quadratic shear flow against the
  closed-form phi-weighted mean (the oracle's own pin, here on the device).
- The fast-bead guard: the sweep updates tiles no bead marked before the
  bead phase ends, which assumes a bead moves less than a cell per step; a
  bead driven past 0.5 cells per step sets FPD_FLAG_FAST_BEAD and from then
  on every tile waits, so the run equals one with the early path off.
- The watchdog: a diverged single instance is reported by fpd_sync.
- The staged sweep's bounded wait on its bulk copy: a barrier made to
  expect more bytes than arrive is given up on, flagged and reported, and
  the context stays usable.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2212_14153_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
THREADS = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def fpd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14153_gb300 import build, fpd as binding
    build.build()
    return binding


# ------------------------------------------------------------ a9: diagnostics
def test_diag_mass_and_momentum_equal_oracle_totals(fpd):
    # forced (body force), moving unequal walls, two fibers with beads:
    # sum_x f and sum_x f c of the GPU's FP64 reduction against the oracle's
    rng = np.random.default_rng(123)
    cfg = wl.random_fiber(rng, 96, 48, n_beads=6, a=2.0, xi=0.5, n_fibers=2, gx=2e-6, gy=-1e-6)
    cfg.update(u_bottom=-0.004, u_top=0.012)
    g = fpd.Simulation(cfg)
    o = oracle.Sim(dict(cfg, threads=THREADS))
    N = cfg["nx"] * cfg["ny"]
    for n in (0, 1, 37, 300):
        g.step(n - int(g.diag()[3]))
        o.step(n - o.nstep)
        d = g.diag()
        t = o.totals()
        assert d[3] == n
        assert abs(d[0] - t[0]) < 1e-12 * N, (n, d, t)
        # momentum scale: N U; both are far above the rounding floor here
        pscale = N * 0.012
        assert abs(d[1] - t[1]) < 1e-12 * pscale and abs(d[2] - t[2]) < 1e-12 * pscale, (n, d, t)
        assert n == 0 or abs(t[1]) > 1e-3 * pscale     # a real signal, not rounding
    nd = np.zeros(4)
    fpd.fpd_diag_noalloc(g.h, nd)
    assert np.allclose(nd[:3], g.diag()[:3], rtol=1e-13, atol=0)


# ------------------------------------------------------------ Eq. 5 on the device
def _phi_moments(a, xi):
    mpmath = pytest.importorskip("mpmath")
    sig = xi / 2.0
    z = -mpmath.e ** (a / sig)
    i1 = -sig ** 2 * mpmath.polylog(2, z)
    i3 = -6 * sig ** 4 * mpmath.polylog(4, z)
    return float(2 * math.pi * i1), float(0.5 * i3 / i1)


@pytest.mark.parametrize("precision,tol", [(0, 5e-8), (1, 2e-6), (2, 1e-2)])
def test_bead_velocity_in_quadratic_shear_matches_closed_form(fpd, precision, tol):
    # V_x = c ((R_y - y0)^2 + <(y - R_y)^2>_phi) for u_x = c (y - y0)^2 (Eq. 5;
    # the closed form and its lattice-sum accuracy, < 1e-8 here, are derived in
    # the oracle's pin of the same case).  FP32 paths: phi and u in FP32
    # (relative rounding ~1e-7 per term) with compensated sums; FP16 storage
    # rounds each population's deviation to 2^-11 of its plane scale.
    nx = ny = 96
    a, xi, c, y0 = 10.0, 2.0, 3e-6, 40.2
    cfg = dict(wl.couette_only(nx, ny, u=0.0, nu=0.1, init_couette=0, precision=precision), periodic_y=1,
               n_beads=1, n_fibers=1, a=a, xi=xi, phi_cut=12.0, k_s=0.0, k_b=0.0, stiffness_K=0.0, k_ev=0.0,
               centres=[[48.3, 47.7]], theta0=[0.0])
    s = fpd.Simulation(cfg)
    s.step(1)
    R = s.beads()[0][0].copy()
    y = np.arange(ny) + 0.5
    f = np.stack([oracle.feq(1.0, c * (yy - y0) ** 2, 0.0) for yy in y], axis=1)
    s.set_populations(np.repeat(f[:, :, None], nx, axis=2))
    s.step(1)
    R1, V, F, S = s.beads()
    area, m2 = _phi_moments(a, xi)
    expect = c * ((R[1] - y0) ** 2 + m2)
    print(f"precision {precision}: V_x / closed form - 1 = {V[0, 0] / expect - 1:.2e}, S {S[0] / area - 1:.2e}")
    assert abs(S[0] / area - 1) < max(tol, 5e-8)
    assert abs(V[0, 0] / expect - 1) < tol
    assert abs(V[0, 1]) < max(tol, 1e-12) * abs(V[0, 0])


# ------------------------------------------------------------ fast-bead guard
def _driven(precision, F0, L=48):
    return dict(nx=L, ny=L, u_bottom=0.0, u_top=0.0, nu_f=0.1, re=1.0, visc_ratio=20.0, xi=0.5, a=2.0,
                n_beads=1, n_fibers=1, k_s=0.0, k_b=0.0, stiffness_K=0.0, k_ev=0.0, phi_cut=8.0, collision=0,
                s_e=1.64, s_eps=1.54, s_q=1.9, init_couette=0, periodic_y=1, bead_fx=F0, bead_fy=0.0,
                gx=-F0 / (L * L), gy=0.0, centres=[[20.3, 24.6]], theta0=[0.0], precision=precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_fast_bead_sets_flag_and_keeps_results_of_the_waiting_path(fpd, precision, monkeypatch):
    # F_0 = 1 drives the bead past 0.5 cells per step at step ~285 (the
    # oracle's run of this case: V_x 0.44 at step 200, 0.57 at step 400; at
    # F_0 = 2 the over-driven flow turns unsteady and, in FP32, non-finite);
    # the guard must flag it, and the run must equal, bit for bit, the one in
    # which no tile ever updates early
    cfg = _driven(precision, 1.0)
    a = fpd.Simulation(cfg)
    monkeypatch.setenv("FPD_NO_EARLY_COLD", "1")
    b = fpd.Simulation(cfg)
    monkeypatch.delenv("FPD_NO_EARLY_COLD")
    vmax = 0.0
    for s in (a, b):
        for chunk in (1, 100, 3, 64, 32, 200):   # direct steps and captured chunks
            s.step(chunk)
            if s is a:
                vmax = max(vmax, float(np.abs(s.beads()[1]).max()))
    assert vmax >= 0.5
    assert a.flags() & fpd.FPD_FLAG_FAST_BEAD and b.flags() & fpd.FPD_FLAG_FAST_BEAD
    fa, fb = a.populations(), b.populations()
    assert np.array_equal(fa, fb, equal_nan=True)
    for x, y in zip(a.beads(), b.beads()):
        assert np.array_equal(x, y, equal_nan=True)


def test_slow_bead_leaves_flags_clear(fpd):
    # the same bead driven ten times more gently stays far below the limit
    s = fpd.Simulation(_driven(0, 0.2))
    s.step(300)
    assert float(np.abs(s.beads()[1]).max()) < 0.2
    assert s.flags() == 0
    s.sync()


# ------------------------------------------------------------ watchdog
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_watchdog_reports_a_diverged_instance_at_sync(fpd, precision):
    cfg = wl.couette_only(64, 32, u=0.01, nu=0.2, precision=precision)
    cfg["gx"] = 1e300
    s = fpd.Simulation(cfg)
    s.step(100)          # no watchdog pass yet: the first runs after 1024 steps
    s.sync()
    assert s.flags() == 0
    s.step(1000)
    assert s.flags() & fpd.FPD_FLAG_NONFINITE
    with pytest.raises(fpd.FpdError) as e:
        s.sync()
    assert e.value.code == fpd.FPD_ENAN
    s.close()
    good = fpd.Simulation(wl.couette_only(64, 32, u=0.01, nu=0.2, precision=precision))
    good.step(1100)
    good.sync()
    assert good.flags() == 0


# ------------------------------------------------- staged sweep: bounded wait
@pytest.mark.parametrize("precision", [1, 2])
def test_staged_copy_wait_runs_out_and_is_reported(fpd, precision, monkeypatch):
    # the staged sweep (variant 3) waits a bounded time for the bulk copy of
    # its block.  FPD_TEST_COPY_SHORTFALL=1 has each block's barrier expect
    # 16 bytes more than its copy moves, so no wait can complete (the copy
    # itself lands, nothing faults): every CTA of an inner block gives up
    # after 0.1 s, sets FPD_FLAG_COPY_TIMEOUT and ends, and fpd_sync reports
    # FPD_ECUDA.  The context stays usable: fresh instances then run the
    # staged sweep bit for bit like variant 1
    rng = np.random.default_rng(4242 + precision)
    cfg = wl.random_fiber(rng, 160, 150, n_beads=8, a=2.5, xi=1.0, precision=precision)
    monkeypatch.setenv("FPD_TEST_COPY_SHORTFALL", "1")
    bad = fpd.Simulation(cfg)
    monkeypatch.delenv("FPD_TEST_COPY_SHORTFALL")
    bad.set_tuning(3)
    bad.step(1)
    assert bad.flags() & fpd.FPD_FLAG_COPY_TIMEOUT
    with pytest.raises(fpd.FpdError) as e:
        bad.sync()
    assert e.value.code == fpd.FPD_ECUDA
    bad.close()
    a, b = fpd.Simulation(cfg), fpd.Simulation(cfg)
    a.set_tuning(3)
    b.set_tuning(1)
    a.step(40)
    b.step(40)
    a.sync()
    assert a.flags() == 0
    assert np.array_equal(a.populations(), b.populations())
