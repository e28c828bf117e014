"""FP64 CPU oracle of the extended-FPD MRT-LBM step (arXiv 2212.14153).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(the CUDA library and its binding) never does.  It shares no code with the
CUDA path.  The arithmetic lives in ``fpd_oracle.c`` (plain C, compiled with
``-ffp-contract=off``); this module only marshals arguments through ctypes.

Parity status per function (what pins each, all in ``tests/test_oracle*.py``):
  moment basis / equilibria / Guo forms  -- closed forms, orthogonality
  MRT collision                           -- equal rates == velocity-space BGK
  streaming + moving-wall bounce-back     -- rest fixed point, exact mass,
                                             linear Couette steady state
  forcing + wall location                 -- body-force Poiseuille parabola
  bead forces (Eqs. 11-12, ext. volume)   -- finite differences of the energy,
                                             zero net force and torque
  spreading / reduction (Eqs. 4-5)        -- sum of f = sum of F_i, uniform
                                             velocity gives V_i = U exactly
  coupled step                            -- Jeffery period of a stiff fiber
  sandwich layers (Eq. 14)                -- steady variable-viscosity
                                             Couette closed form, 2nd order
  periodic y, driven bead, eps_v          -- Hasimoto's drag of a periodic
                                             array of discs; eps_v -> 0 for a
                                             uniformly translating fluid
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fpd_oracle.c")
_LIB = os.path.join(_HERE, "libfpd_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libfpd_oracle.so`` (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("u_bottom", ctypes.c_double), ("u_top", ctypes.c_double),
        ("nu_f", ctypes.c_double), ("re", ctypes.c_double),
        ("visc_ratio", ctypes.c_double), ("xi", ctypes.c_double),
        ("a", ctypes.c_double),
        ("n_beads", ctypes.c_int32), ("n_fibers", ctypes.c_int32),
        ("k_s", ctypes.c_double), ("k_b", ctypes.c_double),
        ("stiffness_K", ctypes.c_double), ("k_ev", ctypes.c_double),
        ("phi_cut", ctypes.c_double), ("gx", ctypes.c_double),
        ("gy", ctypes.c_double), ("collision", ctypes.c_int32),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double),
        ("s_q", ctypes.c_double), ("init_couette", ctypes.c_int32),
        ("threads", ctypes.c_int32), ("sandwich_zl", ctypes.c_double),
        ("sandwich_zr", ctypes.c_double), ("periodic_y", ctypes.c_int32),
        ("bead_fx", ctypes.c_double), ("bead_fy", ctypes.c_double),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(OrcParams)
            sigs = {
                "orc_create": (ctypes.c_void_p, [P, _DP, _DP, _DP]),
                "orc_destroy": (None, [ctypes.c_void_p]),
                "orc_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_long]),
                "orc_nstep": (ctypes.c_long, [ctypes.c_void_p]),
                "orc_fields": (None, [ctypes.c_void_p, _DP, _DP, _DP]),
                "orc_get_populations": (None, [ctypes.c_void_p, _DP]),
                "orc_set_populations": (None, [ctypes.c_void_p, _DP]),
                "orc_overlay_fields": (None, [ctypes.c_void_p, _DP, _DP, _DP]),
                "orc_beads": (None, [ctypes.c_void_p, _DP, _DP, _DP, _DP]),
                "orc_totals": (None, [ctypes.c_void_p, _DP]),
                "orc_derived": (None, [ctypes.c_void_p, _DP]),
                "orc_moment_matrix": (None, [_DP]),
                "orc_inverse_moment_matrix": (None, [_DP]),
                "orc_feq": (None, [ctypes.c_double] * 3 + [_DP]),
                "orc_meq": (None, [ctypes.c_double] * 3 + [_DP]),
                "orc_guo_velocity": (None, [ctypes.c_double] * 4 + [_DP]),
                "orc_guo_moment": (None, [ctypes.c_double] * 4 + [_DP]),
                "orc_rates": (None, [ctypes.c_int] + [ctypes.c_double] * 4 + [_DP]),
                "orc_collide_mrt": (None, [_DP, ctypes.c_double, ctypes.c_double, _DP, _DP]),
                "orc_collide_bgk": (None, [_DP, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, _DP]),
                "orc_bead_forces": (None, [P, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, _DP, _DP]),
                "orc_bead_energy": (ctypes.c_double, [P, ctypes.c_double, ctypes.c_double,
                                                      ctypes.c_double, _DP]),
                "orc_phi": (ctypes.c_double, [ctypes.c_double] * 8),
                "orc_internal_flow": (None, [ctypes.c_void_p, _DP]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


DEFAULTS = dict(
    nx=16, ny=16, u_bottom=0.0, u_top=0.0, nu_f=-1.0, re=1.0, visc_ratio=50.0,
    xi=1.0, a=2.0, n_beads=0, n_fibers=0, k_s=-1.0, k_b=0.0, stiffness_K=0.0,
    k_ev=-1.0, phi_cut=8.0, gx=0.0, gy=0.0, collision=0, s_e=1.64, s_eps=1.54,
    s_q=1.9, init_couette=1, threads=1, sandwich_zl=0.0, sandwich_zr=0.0,
    periodic_y=0, bead_fx=0.0, bead_fy=0.0,
)


def make_params(**kw) -> OrcParams:
    """Oracle parameter struct; unknown keys (e.g. centres) are ignored."""
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k in d:
            d[k] = v
    return OrcParams(**d)


# ---------------------------------------------------------------- helpers
def moment_matrix() -> np.ndarray:
    out = np.zeros(81)
    _load().orc_moment_matrix(_ptr(out))
    return out.reshape(9, 9)


def inverse_moment_matrix() -> np.ndarray:
    out = np.zeros(81)
    _load().orc_inverse_moment_matrix(_ptr(out))
    return out.reshape(9, 9)


def feq(rho, ux, uy) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_feq(rho, ux, uy, _ptr(out))
    return out


def meq(rho, ux, uy) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_meq(rho, ux, uy, _ptr(out))
    return out


def guo_velocity(ux, uy, Fx, Fy) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_guo_velocity(ux, uy, Fx, Fy, _ptr(out))
    return out


def guo_moment(ux, uy, Fx, Fy) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_guo_moment(ux, uy, Fx, Fy, _ptr(out))
    return out


def rates(collision, nu, s_e=1.64, s_eps=1.54, s_q=1.9) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_rates(collision, nu, s_e, s_eps, s_q, _ptr(out))
    return out


def collide_mrt(f, Fx, Fy, s) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.zeros(9)
    _load().orc_collide_mrt(_ptr(f), Fx, Fy, _ptr(s), _ptr(out))
    return out


def collide_bgk(f, Fx, Fy, tau) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(9)
    _load().orc_collide_bgk(_ptr(f), Fx, Fy, tau, _ptr(out))
    return out


def bead_forces(R, n_beads, n_fibers, a, k_s, k_b, k_ev, nx=10**6, **extra) -> np.ndarray:
    p = make_params(nx=nx, n_beads=n_beads, n_fibers=n_fibers, a=a, **extra)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
    F = np.zeros_like(R)
    _load().orc_bead_forces(ctypes.byref(p), k_s, k_b, k_ev, _ptr(R), _ptr(F))
    return F.reshape(-1, 2)


def bead_energy(R, n_beads, n_fibers, a, k_s, k_b, k_ev, nx=10**6, **extra) -> float:
    p = make_params(nx=nx, n_beads=n_beads, n_fibers=n_fibers, a=a, **extra)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
    return _load().orc_bead_energy(ctypes.byref(p), k_s, k_b, k_ev, _ptr(R))


def phi(a, xi, rcut, nx, xc, yc, Rx, Ry) -> float:
    return _load().orc_phi(a, xi, rcut, nx, xc, yc, Rx, Ry)


# ---------------------------------------------------------------- simulation
class Sim:
    """One oracle simulation.  ``cfg`` holds the same keys as the CUDA
    library's parameter struct; ``centres`` (n_fibers x 2) and ``theta0``
    (radians, n_fibers) place the fibers, or ``R0`` (n_beads*n_fibers x 2)."""

    def __init__(self, cfg: dict, R0=None):
        self.cfg = dict(cfg)
        self.p = make_params(**cfg)
        self.nx, self.ny = self.p.nx, self.p.ny
        self.nb = self.p.n_beads * self.p.n_fibers
        lib = _load()
        nf = max(self.p.n_fibers, 1)
        cen = np.ascontiguousarray(cfg.get("centres", np.zeros((nf, 2))), dtype=np.float64).reshape(-1)
        th = np.ascontiguousarray(cfg.get("theta0", np.zeros(nf)), dtype=np.float64).reshape(-1)
        if R0 is not None:
            R0 = np.ascontiguousarray(R0, dtype=np.float64).reshape(-1)
            h = lib.orc_create(ctypes.byref(self.p), _ptr(R0), None, None)
        else:
            h = lib.orc_create(ctypes.byref(self.p), None, _ptr(cen), _ptr(th))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = ctypes.c_void_p(h)
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_destroy(h)
            self._h = None

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))

    @property
    def nstep(self) -> int:
        return self._lib.orc_nstep(self._h)

    def fields(self):
        ux = np.zeros((self.ny, self.nx)); uy = np.zeros_like(ux); rho = np.zeros_like(ux)
        self._lib.orc_fields(self._h, _ptr(ux), _ptr(uy), _ptr(rho))
        return ux, uy, rho

    def populations(self) -> np.ndarray:
        f = np.zeros((9, self.ny, self.nx))
        self._lib.orc_get_populations(self._h, _ptr(f))
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx)
        self._lib.orc_set_populations(self._h, _ptr(f))

    def overlay_fields(self):
        fx = np.zeros((self.ny, self.nx)); fy = np.zeros_like(fx); nu = np.zeros_like(fx)
        self._lib.orc_overlay_fields(self._h, _ptr(fx), _ptr(fy), _ptr(nu))
        return fx, fy, nu

    def beads(self):
        n = max(self.nb, 1)
        R = np.zeros((n, 2)); V = np.zeros((n, 2)); F = np.zeros((n, 2)); S = np.zeros(n)
        self._lib.orc_beads(self._h, _ptr(R), _ptr(V), _ptr(F), _ptr(S))
        k = self.nb
        return R[:k], V[:k], F[:k], S[:k]

    def totals(self):
        out = np.zeros(3)
        self._lib.orc_totals(self._h, _ptr(out))
        return out

    def internal_flow(self) -> np.ndarray:
        """eps_v of every bead (Sec. 3.2): sum phi (v - V)^2 / sum phi."""
        out = np.zeros(max(self.nb, 1))
        self._lib.orc_internal_flow(self._h, _ptr(out))
        return out[:self.nb]

    def derived(self) -> dict:
        out = np.zeros(7)
        self._lib.orc_derived(self._h, _ptr(out))
        keys = ["nu_f", "k_s", "k_b", "k_ev", "l0", "rcut", "gamma_dot"]
        return dict(zip(keys, out.tolist()))


def fiber_angle(R: np.ndarray, n_beads: int, fiber: int = 0) -> float:
    """Orientation of the end-to-end vector R_N - R_1 (radians, atan2)."""
    Rf = R[fiber * n_beads:(fiber + 1) * n_beads]
    d = Rf[-1] - Rf[0]
    return math.atan2(d[1], d[0])
