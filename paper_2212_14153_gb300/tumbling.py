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


def run_tracks(configs: list[dict], steps: int, sample_every: int, precision: int = 1,
               stream=None) -> list[Track]:
    """Advance every configuration together on the batched engine for
    `steps` time steps, sampling each fiber's orientation and end-to-end
    ratio every `sample_every` steps (the shape-diagram sweeps of Sec. 4)."""
    from . import fpd
    l0 = [2.0 * c["a"] for c in configs]
    cells = sum(int(c["nx"]) * int(c["ny"]) for c in configs)
    es = {0: 8, 1: 4, 2: 2}[precision]
    pool = 9 * es * (cells + 64 * sum(int(c["ny"]) for c in configs)) + 4096 * len(configs)
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
