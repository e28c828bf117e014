"""Tumbling sweeps and shape regimes on the batched engine (Sec. 4).

Loose physical checks (the paper's resolution is not stated, so its figure
values are context, not pins): the Fig. 7 configuration at three stiffnesses
and a Reynolds-number sweep of a rigid fiber.  Run with -s to see the
measured periods and regimes.
"""
import math

import numpy as np
import pytest

from paper_2212_14153_gb300 import studies
from paper_2212_14153_gb300 import tumbling as tb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14153_gb300 import build
    build.build()


def fiber_case(K, C, Re_ps, theta0=math.radians(80.0)):
    return tb.tumbling_case(K, C, Re_ps, N=10, a=2.0, U=0.02, theta0=theta0, r_eta=100.0)


def test_fig7_stiffness_regimes():
    cases = [fiber_case(K, 0.5, 1.5) for K in (3.3, 0.33, 3.3e-5)]
    g = cases[0][1]
    steps = int(2.6 * tb.jeffery_half_period(0.1, g))
    tracks = tb.run_tracks([c for c, _ in cases], steps, 200)
    mins, labels = [], []
    for (cfg, _), tr in zip(cases, tracks):
        t, th, e2e = tr.arrays()
        lab = tb.classify(t, th, e2e, g)
        hp = tb.half_periods(t, th)
        print(f"K = {cfg['stiffness_K']:g}: regime {lab}, min end-to-end {e2e.min():.3f}, "
              f"half-periods (gamma_dot T) {np.round(hp * g, 2)}")
        mins.append(e2e.min())
        labels.append(lab)
    assert labels[0] in ("jeffery", "jeffery-stuck")     # the stiff fiber stays straight
    assert mins[0] > 0.97
    assert mins[0] >= mins[1] >= mins[2]                  # softer fibers bend more
    assert mins[2] < 0.9


def test_rigid_period_grows_with_reynolds():
    # Fig. 5b: at weak confinement the period of a rigid fiber grows with Re_ps
    res = [0.25, 1.0, 1.75]
    cases = [fiber_case(3.3, 0.2, r, theta0=math.pi / 2) for r in res]
    g = cases[0][1]
    steps = int(1.6 * tb.jeffery_half_period(0.12, g))
    tracks = tb.run_tracks([c for c, _ in cases], steps, 100)
    periods = []
    for r, tr in zip(res, tracks):
        t, th, e2e = tr.arrays()
        # first full 180-degree turn from the vertical start
        k = np.argmax(th <= -math.pi / 2)
        assert k > 0, "did not complete a half turn"
        T = t[k - 1] + (-math.pi / 2 - th[k - 1]) / (th[k] - th[k - 1]) * (t[k] - t[k - 1])
        r_fit, resid = tb.jeffery_fit(t[t > 0.05 * steps], th[t > 0.05 * steps], g)
        periods.append(T)
        print(f"Re_ps = {r}: gamma_dot T_180 = {T * g:.2f}, Jeffery fit r_e = {r_fit:.3f} (rms {resid:.3f})")
    assert periods[0] < periods[1] < periods[2]


def test_rigid_critical_reynolds_and_stuck_angle():
    # Fig. 5b / Fig. 6b, r_c = 0.1, C = 0.2: the period diverges as
    # (Re_cr - Re_ps)^-1/2 with Re_cr ~ 2.2, and at Re_ps = 6 the fiber
    # sticks at ~20.4 degrees (tests/golden).  Loose pins: the paper's
    # resolution is unstated
    from conftest import paper_value
    re_cr = paper_value("rigid_re")["x_cr"]
    stuck = paper_value("stuck_angle_deg")["value"]
    out = studies.sweep("rigid-re", values=[0.25, 1.0, 1.5, 1.75, 2.0, 6.0])
    rows = out["rows"]
    for r in rows:
        print(f"Re_ps = {r['x']}: gamma_dot T = {r['gT']:.2f}, stuck at {r['stuck_deg']:.2f} deg")
    fit = out["fit_paper_beta"]
    print("fit (beta = 1/2):", fit, "free beta:", out.get("fit_free_beta"))
    T = [r["gT"] for r in rows[:5]]
    assert all(np.isfinite(T)) and np.all(np.diff(T) > 0)
    assert abs(fit["x_cr"] / re_cr - 1) < 0.15 and fit["rms"] < 0.03
    assert not np.isfinite(rows[5]["gT"]) and abs(rows[5]["stuck_deg"] - stuck) < 5.0
