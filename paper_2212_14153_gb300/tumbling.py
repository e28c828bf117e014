"""Fiber orientation, tumbling periods and shape regimes (Sec. 4 of the paper).

Host-side analysis of bead trajectories produced by the CUDA library (single
instances or a batch).  A fiber is head-tail symmetric, so its orientation
theta (the angle of R_N - R_1 to +x) is tracked modulo pi and unwrapped in
time.  The tumbling period T is the time of a 180-degree rotation (Sec. 4.2);
the angular velocity of a rigid fiber follows Jeffery's orbit (Eq. 19)
    omega = (gamma_dot / 2) [A cos 2 theta - 1],  A = (1 - r^2) / (1 + r^2),
and the shape regimes of Sec. 4.3 are told apart by the end-to-end length:
  jeffery  - tumbles and stays straight,
  s-turn   - tumbles, bends into an S and straightens again each turn,
  s-coiled - tumbles folded (stays short),
  stuck    - stops rotating (jeffery-stuck if straight, s-stuck if bent).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def orientation(R: np.ndarray, n_beads: int, fiber: int = 0) -> float:
    """Angle of the end-to-end vector of one fiber (radians, (-pi, pi])."""
    Rf = R[fiber * n_beads:(fiber + 1) * n_beads]
    d = Rf[-1] - Rf[0]
    return math.atan2(float(d[1]), float(d[0]))


def end_to_end_ratio(R: np.ndarray, n_beads: int, l0: float, fiber: int = 0) -> float:
    """|R_N - R_1| over the straight length (N - 1) l0."""
    Rf = R[fiber * n_beads:(fiber + 1) * n_beads]
    return float(np.linalg.norm(Rf[-1] - Rf[0]) / ((n_beads - 1) * l0))


@dataclass
class Track:
    """Unwrapped orientation and end-to-end ratio sampled in time."""
    t: list = field(default_factory=list)
    theta: list = field(default_factory=list)
    e2e: list = field(default_factory=list)

    def add(self, t: float, theta: float, e2e: float):
        if self.theta:
            prev = self.theta[-1]
            d = theta - prev
            d -= math.pi * round(d / math.pi)  # nearest head-tail-equivalent angle
            theta = prev + d
        self.t.append(float(t))
        self.theta.append(float(theta))
        self.e2e.append(float(e2e))

    def arrays(self):
        return np.array(self.t), np.array(self.theta), np.array(self.e2e)


def half_periods(t: np.ndarray, theta: np.ndarray, phase: float = math.pi / 2) -> np.ndarray:
    """Durations of successive 180-degree turns: times between crossings of
    phase + k pi (k integer) by the unwrapped angle, linearly interpolated."""
    k = np.floor((theta - phase) / math.pi)
    cross = []
    for i in range(1, len(t)):
        if k[i] != k[i - 1]:
            level = phase + math.pi * max(k[i], k[i - 1])
            a, b = theta[i - 1], theta[i]
            if b == a:
                continue
            cross.append(t[i - 1] + (level - a) / (b - a) * (t[i] - t[i - 1]))
    return np.diff(np.array(cross))


def angular_velocity(t: np.ndarray, theta: np.ndarray) -> np.ndarray:
    return np.gradient(theta, t)


def jeffery_fit(t: np.ndarray, theta: np.ndarray, gamma_dot: float) -> tuple[float, float]:
    """Least-squares fit of Eq. 19 to omega(theta): returns (r_e, rms
    residual / gamma_dot).  A is fitted from omega + g/2 = (g/2) A cos 2 theta."""
    om = angular_velocity(t, theta)
    c2 = 0.5 * gamma_dot * np.cos(2 * theta)
    A = float(np.sum((om + 0.5 * gamma_dot) * c2) / np.sum(c2 * c2))
    A = min(max(A, -0.999999), 0.999999)
    resid = om - 0.5 * gamma_dot * (A * np.cos(2 * theta) - 1)
    return math.sqrt((1 - A) / (1 + A)), float(np.sqrt(np.mean(resid ** 2)) / gamma_dot)


def jeffery_half_period(r_e: float, gamma_dot: float) -> float:
    """180-degree period of Eq. 19: pi (r + 1/r) / gamma_dot."""
    return math.pi * (r_e + 1.0 / r_e) / gamma_dot


def jeffery_angle(t: np.ndarray, theta0: float, r_e: float, gamma_dot: float) -> np.ndarray:
    """Closed-form integral of Eq. 19 (clockwise tumbling for gamma_dot > 0):
    tan theta = r tan phi with phi = phi0 - gamma_dot r t / (1 + r^2); theta
    is unwrapped along phi (both lie in the same quadrant)."""
    phi0 = math.atan2(math.sin(theta0), r_e * math.cos(theta0))
    phi = phi0 - gamma_dot * r_e * np.asarray(t, dtype=float) / (1 + r_e * r_e)
    return phi + (np.arctan2(r_e * np.sin(phi), np.cos(phi)) - np.arctan2(np.sin(phi), np.cos(phi)))


def classify(t: np.ndarray, theta: np.ndarray, e2e: np.ndarray, gamma_dot: float,
             straight: float = 0.97, coiled: float = 0.9, stuck_deg: float = 5.0) -> str:
    """Shape regime of Sec. 4.3 from an orientation / end-to-end history.

    The fiber is stuck if over the last third of the record it turned by less
    than stuck_deg degrees.  A tumbling fiber is 'jeffery' if it never bends
    (end-to-end ratio >= straight), 's-turn' if it bends and straightens again
    within each turn after the first, 's-coiled' if after its first turn it
    stays below `coiled` most of the time."""
    n = len(t)
    tail = slice(2 * n // 3, n)
    turned = abs(theta[tail][-1] - theta[tail][0])
    if math.degrees(turned) < stuck_deg:
        return "jeffery-stuck" if e2e[tail].min() >= straight else "s-stuck"
    if e2e.min() >= straight:
        return "jeffery"
    hp = half_periods(t, theta)
    if len(hp) == 0:
        return "s-coiled" if np.mean(e2e[tail] < coiled) > 0.5 else "s-turn"
    # after the first 180-degree turn
    first = t[0] + hp[0] if len(hp) else t[0]
    later = t >= first
    if np.mean(e2e[later] < coiled) > 0.5:
        return "s-coiled"
    return "s-turn"


def critical_fit(x: np.ndarray, T: np.ndarray, beta: float = 0.5) -> tuple[float, float, float]:
    """Fit of the divergence law of Secs. 4.2-4.3, gamma_dot T = A (x_cr - x)^-beta
    (x = Re_ps or the confinement C), for a given exponent beta.  With beta
    fixed, T^(-1/beta) = c (x_cr - x) is a straight line in x, fitted by least
    squares.  Returns (x_cr, T0, rms relative residual of T), T0 being the
    law extrapolated to x = 0 (the paper's normalisation)."""
    x = np.asarray(x, dtype=float)
    T = np.asarray(T, dtype=float)
    y = T ** (-1.0 / beta)
    slope, icpt = np.polyfit(x, y, 1)
    c = -slope
    x_cr = icpt / c
    T0 = icpt ** (-beta)
    pred = (c * (x_cr - x)) ** (-beta)
    return float(x_cr), float(T0), float(np.sqrt(np.mean((pred / T - 1.0) ** 2)))


def critical_fit_beta(x: np.ndarray, T: np.ndarray, betas=None) -> tuple[float, float, float, float]:
    """As critical_fit with the exponent also fitted (scanned over `betas`,
    default 0.05 .. 2 in steps of 0.01): returns (x_cr, T0, beta, rms)."""
    betas = np.arange(0.05, 2.0001, 0.01) if betas is None else betas
    best = None
    for b in betas:
        with np.errstate(invalid="ignore", divide="ignore"):
            x_cr, T0, rms = critical_fit(x, T, float(b))
        if np.isfinite(rms) and x_cr > np.max(x) and (best is None or rms < best[3]):
            best = (x_cr, T0, float(b), rms)
    if best is None:
        raise ValueError("no exponent gives a critical point beyond the data")
    return best


def tumbling_case(K: float, C: float, Re_ps: float, N: int = 10, a: float = 2.0, U: float = 0.02,
               theta0: float = math.pi / 2, r_eta: float = 100.0, r_xi: float = 0.125,
               lx_over_d: float = 25.0) -> tuple[dict, float]:
    """Configuration of the Sec. 4 tumbling runs: one fiber of N beads of
    diameter d = 2a (l_c = N d, r_c = 1/N) centred between walls at -U and
    +U, H = l_c / C, L_x = lx_over_d d, Re = 4 Re_ps (Eq. 18), xi = r_xi d.
    Returns (config, shear rate 2U/H)."""
    d = 2.0 * a
    lc = d * N
    H = int(round(lc / C))
    Lx = int(round(lx_over_d * d))
    cfg = dict(nx=Lx, ny=H, u_bottom=-U, u_top=U, nu_f=-1.0, re=4.0 * Re_ps, visc_ratio=r_eta,
               xi=r_xi * d, a=a, n_beads=N, n_fibers=1, stiffness_K=K, k_s=-1.0, k_b=0.0, k_ev=-1.0,
               phi_cut=8.0, gx=0.0, gy=0.0, collision=0, s_e=1.64, s_eps=1.54, s_q=1.9,
               init_couette=1, centres=[[Lx / 2.0, H / 2.0]], theta0=[theta0])
    return cfg, 2.0 * U / H


@dataclass
class PeriodResult:
    T: float             # steps per steady 180-degree turn (inf if none)
    stuck_deg: float     # orientation (degrees, in (-90, 90]) of a stuck fiber, else nan
    track: Track


def _crossing(t, th, level):
    """First time the unwrapped angle falls to `level` (linear interpolation)."""
    k = int(np.argmax(th <= level))
    if th[k] > level:
        return None
    if k == 0:
        return float(t[0])
    return float(t[k - 1] + (level - th[k - 1]) / (th[k] - th[k - 1]) * (t[k] - t[k - 1]))


def measure_periods(configs: list[dict], max_steps: int, sample_every: int = 200, precision: int = 1,
                    stuck_window: int | None = None, stuck_deg: float = 1.0,
                    stream=None) -> list[PeriodResult]:
    """Tumbling period T of every configuration (Sec. 4.2: the time of a
    180-degree rotation), measured on the batched engine.

    The first half turn after placement carries the start-up transient, so T
    is taken between the first two crossings of the fiber's orientation
    through theta0 - pi/2 and theta0 - 3 pi/2 (for theta0 = pi/2: from
    horizontal to horizontal).  An instance leaves the batch as soon as its
    period is measured, or when over the last `stuck_window` steps (default
    max_steps / 5) it has turned by less than `stuck_deg` degrees (stuck,
    Secs. 4.2-4.3), or at max_steps (T = inf), or once its beads are no
    longer finite (T = nan)."""
    from . import fpd
    W = stuck_window or max(sample_every, max_steps // 5)
    cells = sum(int(c["nx"]) * int(c["ny"]) for c in configs)
    es = {0: 8, 1: 4, 2: 2}[precision]
    pool = 18 * es * (cells + 64 * sum(int(c["ny"]) for c in configs)) + 4096 * len(configs)
    nbeads = sum(int(c["n_beads"]) * int(c["n_fibers"]) for c in configs)
    b = fpd.Batch(precision, len(configs), pool, nbeads, stream)
    slots = [b.add(dict(c, precision=precision), max_steps) for c in configs]
    tracks = [Track() for _ in configs]
    th0 = [float(c["theta0"][0]) for c in configs]
    res: list[PeriodResult | None] = [None] * len(configs)
    live = set(range(len(configs)))

    def sample(t):
        for i in list(live):
            c = configs[i]
            R = b.beads(slots[i])[0]
            if not np.all(np.isfinite(R)):
                # diverged (an unstable parameter set): no period
                res[i] = PeriodResult(float("nan"), float("nan"), tracks[i])
                live.discard(i)
                b.remove(slots[i])
                continue
            tracks[i].add(t, orientation(R, c["n_beads"]),
                          end_to_end_ratio(R, c["n_beads"], 2.0 * c["a"]))

    sample(0)
    done = 0
    while live and done < max_steps:
        d = b.run(min(sample_every, max_steps - done))
        if d == 0:
            break
        done += d
        sample(done)
        for i in list(live):
            t, th, _ = tracks[i].arrays()
            if len(t) == 0:
                continue
            # orientation is taken modulo pi; align the first sample with theta0
            th = th + math.pi * round((th0[i] - th[0]) / math.pi)
            t1 = _crossing(t, th, th0[i] - math.pi / 2)
            t2 = _crossing(t, th, th0[i] - 1.5 * math.pi) if t1 is not None else None
            if t2 is not None:
                res[i] = PeriodResult(t2 - t1, float("nan"), tracks[i])
            elif t[-1] >= W:
                j = int(np.searchsorted(t, t[-1] - W))
                if abs(th[-1] - th[j]) < math.radians(stuck_deg):
                    ang = math.degrees(th[-1]) % 180.0
                    res[i] = PeriodResult(float("inf"), ang - 180.0 if ang > 90.0 else ang, tracks[i])
            if res[i] is not None:
                live.discard(i)
                b.remove(slots[i])
    for i in live:
        res[i] = PeriodResult(float("inf"), float("nan"), tracks[i])
    b.close()
    return res


def run_tracks(configs: list[dict], steps: int, sample_every: int, precision: int = 1,
               stream=None) -> list[Track]:
    """Advance every configuration together on the batched engine for
    `steps` time steps, sampling each fiber's orientation and end-to-end
    ratio every `sample_every` steps (the shape-diagram sweeps of Sec. 4)."""
    from . import fpd
    l0 = [2.0 * c["a"] for c in configs]
    cells = sum(int(c["nx"]) * int(c["ny"]) for c in configs)
    es = {0: 8, 1: 4, 2: 2}[precision]
    pool = 18 * es * (cells + 64 * sum(int(c["ny"]) for c in configs)) + 4096 * len(configs)
    nbeads = sum(int(c["n_beads"]) * int(c["n_fibers"]) for c in configs)
    b = fpd.Batch(precision, len(configs), pool, nbeads, stream)
    slots = [b.add(dict(c, precision=precision), steps) for c in configs]
    tracks = [Track() for _ in configs]

    def sample(t):
        for c, s, tr, L in zip(configs, slots, tracks, l0):
            R = b.beads(s)[0]
            tr.add(t, orientation(R, c["n_beads"]), end_to_end_ratio(R, c["n_beads"], L))

    sample(0)
    done = 0
    while done < steps:
        d = b.run(min(sample_every, steps - done))
        if d == 0:
            break
        done += d
        sample(done)
    b.close()
    return tracks
