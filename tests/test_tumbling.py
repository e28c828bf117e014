"""Host analysis of tumbling (Sec. 4): orientation tracking, periods, the
Jeffery fit of Eq. 19 and the shape-regime classifier, on analytic and
synthetic histories (no GPU)."""
import math

import numpy as np
import pytest

from paper_2212_14153_gb300 import tumbling as tb


@pytest.mark.parametrize("r_e", [0.1, 0.132, 0.25])
def test_analytic_jeffery_orbit_satisfies_eq19_and_period(r_e):
    g = 5e-4
    T = tb.jeffery_half_period(r_e, g)
    t = np.linspace(0, 3.2 * T, 40001)
    th = tb.jeffery_angle(t, math.pi / 2, r_e, g)
    # the closed form obeys Eq. 19 pointwise
    om = np.gradient(th, t)
    A = (1 - r_e ** 2) / (1 + r_e ** 2)
    pred = 0.5 * g * (A * np.cos(2 * th) - 1)
    assert np.abs(om - pred)[5:-5].max() < 1e-5 * g   # finite-difference derivative
    # every 180-degree turn takes pi (r + 1/r) / gamma_dot
    hp = tb.half_periods(t, th)
    assert len(hp) >= 2
    assert np.allclose(hp, T, rtol=1e-6)
    # the least-squares fit recovers r_e
    r_fit, resid = tb.jeffery_fit(t, th, g)
    assert abs(r_fit / r_e - 1) < 1e-4 and resid < 1e-5


def test_track_unwraps_head_tail_symmetric_angles():
    tr = tb.Track()
    true = np.linspace(1.5, -6.0, 200)          # clockwise through several turns
    for i, a in enumerate(true):
        wrapped = math.atan2(math.sin(a), math.cos(a))
        if i % 3 == 0:
            wrapped = math.atan2(math.sin(a + math.pi), math.cos(a + math.pi))  # reversed end-to-end
        tr.add(i, wrapped, 1.0)
    _, th, _ = tr.arrays()
    assert np.allclose(th - th[0], true - true[0], atol=1e-12)


def test_orientation_and_end_to_end():
    R = np.array([[0.0, 0.0], [4.0, 0.0], [8.0, 4.0]])
    assert math.isclose(tb.orientation(R, 3), math.atan2(4, 8))
    assert math.isclose(tb.end_to_end_ratio(R, 3, 4.0), math.hypot(8, 4) / 8.0)


def _history(theta, e2e):
    t = np.arange(len(theta), dtype=float)
    return t, np.asarray(theta, float), np.asarray(e2e, float)


def test_classifier_regimes():
    g = 1e-3
    t = np.linspace(0, 3 * tb.jeffery_half_period(0.15, g), 3000)
    th = tb.jeffery_angle(t, 1.0, 0.15, g)
    assert tb.classify(t, th, np.full_like(t, 0.995), g) == "jeffery"
    # bends during each turn and straightens again
    e2e = 0.99 - 0.1 * np.sin(th) ** 8
    assert tb.classify(t, th, e2e, g) == "s-turn"
    # folds during the first turn and stays folded
    e2e = np.where(t > t[-1] * 0.2, 0.6, 0.99)
    assert tb.classify(t, th, e2e, g) == "s-coiled"
    # stops turning
    th_stuck = 0.35 + 0.3 * np.exp(-t / (t[-1] * 0.1))
    assert tb.classify(t, th_stuck, np.full_like(t, 0.99), g) == "jeffery-stuck"
    assert tb.classify(t, th_stuck, np.full_like(t, 0.8), g) == "s-stuck"


@pytest.mark.parametrize("law", ["rigid_re", "rigid_c", "flex_re", "flex_c"])
def test_critical_fit_recovers_the_divergence_law(law):
    # gamma_dot T = T0 (1 - x / x_cr)^-beta, sampled below x_cr (the four
    # laws the paper reports, tests/golden)
    from conftest import paper_value
    v = paper_value(law)
    x_cr, beta, T0 = v["x_cr"], v["beta"], v["gT0"]
    x = np.linspace(0.1, 0.9, 7) * x_cr
    T = T0 * (1 - x / x_cr) ** (-beta)
    xc, t0, rms = tb.critical_fit(x, T, beta)
    assert abs(xc / x_cr - 1) < 1e-10 and abs(t0 / T0 - 1) < 1e-10 and rms < 1e-10
    xc, t0, b, rms = tb.critical_fit_beta(x, T)
    assert abs(b - beta) < 1e-9 and abs(xc / x_cr - 1) < 1e-6
    # the wrong exponent leaves a residual and moves the critical point
    xc2, _, rms2 = tb.critical_fit(x, T, beta + 0.3)
    assert rms2 > 1e-3 and abs(xc2 - x_cr) > 1e-3


def test_critical_fit_with_noise_and_without_divergence():
    rng = np.random.default_rng(3)
    x = np.linspace(0.25, 2.0, 8)
    T = 16.0 * (1 - x / 2.4) ** -0.5 * (1 + 0.01 * rng.standard_normal(x.size))
    xc, t0, rms = tb.critical_fit(x, T, 0.5)
    assert abs(xc - 2.4) < 0.05 and abs(t0 - 16.0) < 0.5 and rms < 0.03
    # a period that does not grow has no critical point beyond the data
    with pytest.raises(ValueError):
        tb.critical_fit_beta(x, 20.0 - x)


def test_tumbling_case_geometry():
    cfg, g = tb.tumbling_case(3.3, 0.2, 1.5, N=10, a=2.0, U=0.02)
    d = 4.0
    assert cfg["ny"] == 200 and cfg["nx"] == 100            # H = l_c / C, L_x = 25 d
    assert cfg["re"] == 6.0 and cfg["xi"] == 0.125 * d      # Re = 4 Re_ps, xi = r_xi d
    assert g == 2 * 0.02 / 200
    assert cfg["centres"] == [[50.0, 100.0]]


def test_hasimoto_inversion_and_driven_case():
    from paper_2212_14153_gb300 import studies
    for a, L in ((2.0, 40.0), (8.0, 160.0), (5.0, 30.0)):
        assert abs(studies.hasimoto_radius(studies.hasimoto_drag(a, L), L) / a - 1) < 1e-9
    # dilute limit: 4 pi / (ln(1/sqrt(c)) - 0.738)
    c = math.pi * 1e-4
    assert abs(studies.hasimoto_drag(1.0, 100.0) / (4 * math.pi / (-0.5 * math.log(c) - 0.738)) - 1) < 1e-3
    cfg = studies.driven_case(8.0, 100.0, 0.0625, 0.1)
    L = cfg["nx"]
    assert L == cfg["ny"] == 160 and cfg["periodic_y"] == 1 and cfg["xi"] == 1.0
    assert cfg["gx"] * L * L == pytest.approx(-cfg["bead_fx"], rel=1e-15)   # no net force on the box
