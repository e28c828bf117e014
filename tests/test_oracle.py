"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
moments, the exact discrete steady states of wall-driven and body-force-driven
channel flow, conservation laws, finite differences of the bead-spring energy
(Eq. 9, bending term without the square, which is the energy whose gradient
is Eq. 12), and invariants of Eqs. 4-5.  No test here needs a GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2212_14153_gb300 import workloads as wl

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
CS2 = 1.0 / 3.0


# ------------------------------------------------------------ moment basis
def test_moment_matrix_rows_orthogonal_with_known_norms():
    M = oracle.moment_matrix()
    G = M @ M.T
    # Lallemand-Luo (2000) basis: squared norms of rho,e,eps,jx,qx,jy,qy,pxx,pxy
    assert np.array_equal(np.diag(G), [9, 36, 36, 6, 12, 6, 12, 4, 4])
    assert np.count_nonzero(G - np.diag(np.diag(G))) == 0
    # the conserved rows are the lattice's mass and momentum
    assert np.array_equal(M[0], np.ones(9))
    assert np.array_equal(M[3], CX) and np.array_equal(M[5], CY)
    assert np.allclose(oracle.inverse_moment_matrix() @ M, np.eye(9), atol=1e-15)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.03, 0.02, -0.015), (0.97, -0.05, 0.04)])
def test_equilibrium_velocity_moments(rho, ux, uy):
    f = oracle.feq(rho, ux, uy)
    # zeroth, first and second velocity moments of the discrete equilibrium
    assert math.isclose(f.sum(), rho, rel_tol=1e-15)
    assert np.allclose([f @ CX, f @ CY], [rho * ux, rho * uy], atol=1e-16)
    Pxx, Pyy, Pxy = f @ (CX * CX), f @ (CY * CY), f @ (CX * CY)
    assert np.allclose([Pxx, Pyy, Pxy], [rho * (CS2 + ux * ux), rho * (CS2 + uy * uy), rho * ux * uy],
                       atol=1e-16)
    # velocity-space equilibrium and the moment-space equilibrium agree
    assert np.allclose(oracle.moment_matrix() @ f, oracle.meq(rho, ux, uy), atol=4e-16)


def test_guo_source_moments_and_two_forms_agree():
    rng = np.random.default_rng(7)
    for _ in range(20):
        ux, uy = rng.uniform(-0.05, 0.05, 2)
        Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
        S = oracle.guo_velocity(ux, uy, Fx, Fy)
        # Guo et al. (2002): zero mass source, momentum source F,
        # second moment u F + F u
        assert abs(S.sum()) < 1e-18
        assert np.allclose([S @ CX, S @ CY], [Fx, Fy], atol=1e-18)
        assert np.allclose([S @ (CX * CX), S @ (CY * CY), S @ (CX * CY)],
                           [2 * ux * Fx, 2 * uy * Fy, ux * Fy + uy * Fx], atol=1e-18)
        Sm = oracle.guo_moment(ux, uy, Fx, Fy)
        assert np.allclose(oracle.moment_matrix() @ S, Sm, rtol=0, atol=1e-14 * max(abs(Fx), abs(Fy)))


# ------------------------------------------------------------ collision
def _random_state(rng):
    rho = rng.uniform(0.95, 1.05)
    u = rng.uniform(-0.05, 0.05, 2)
    return oracle.feq(rho, *u) + rng.normal(0, 2e-3, 9)


def test_mrt_with_equal_rates_is_velocity_space_bgk():
    rng = np.random.default_rng(11)
    for tau in (0.51, 0.8, 1.0, 3.0, 40.0):
        for _ in range(10):
            f = _random_state(rng)
            Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
            a = oracle.collide_mrt(f, Fx, Fy, np.full(9, 1.0 / tau))
            b = oracle.collide_bgk(f, Fx, Fy, tau)
            assert np.abs(a - b).max() <= 1e-14


def test_collision_conserves_mass_and_adds_force_to_momentum():
    rng = np.random.default_rng(12)
    for coll in (0, 1):
        for nu in (0.01, 0.1, 0.5, 25.0):
            s = oracle.rates(coll, nu)
            f = _random_state(rng)
            Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
            out = oracle.collide_mrt(f, Fx, Fy, s)
            assert abs(out.sum() - f.sum()) < 1e-15
            assert np.allclose([out @ CX - f @ CX, out @ CY - f @ CY], [Fx, Fy], atol=1e-16)


def test_rates_of_conserved_moments_do_not_matter():
    rng = np.random.default_rng(13)
    f = _random_state(rng)
    s = oracle.rates(0, 0.2)
    base = oracle.collide_mrt(f, 3e-4, -2e-4, s)
    for srho, sj in [(0.3, 0.7), (1.9, 1.2), (1.0, 0.01)]:
        s2 = s.copy()
        s2[0] = srho
        s2[3] = s2[5] = sj
        assert np.abs(oracle.collide_mrt(f, 3e-4, -2e-4, s2) - base).max() < 1e-16


def test_magic_rates_pairing_and_shear_rate():
    for nu in (0.01, 0.2, 1.0, 25.6):
        s = oracle.rates(0, nu)
        # nu = c_s^2 (1/s_nu - 1/2)
        assert math.isclose(CS2 * (1 / s[7] - 0.5), nu, rel_tol=1e-14)
        assert s[7] == s[8] == s[1] == s[2]
        assert math.isclose((1 / s[7] - 0.5) * (1 / s[4] - 0.5), 3.0 / 16.0, rel_tol=1e-13)


# ------------------------------------------------------------ lattice
def test_rest_equilibrium_is_fixed_point():
    cfg = wl.couette_only(20, 12, u=0.0, nu=0.1, init_couette=0)
    s = oracle.Sim(cfg)
    s.step(500)
    w = oracle.feq(1.0, 0.0, 0.0)
    assert np.abs(s.populations() - w[:, None, None]).max() <= 4e-16


def test_linear_couette_is_exact_steady_state():
    H = 20
    y = np.arange(H) + 0.5
    exact = -0.01 + 0.02 * y / H
    # magic MRT pairing and BGK: exact to round-off.  The constant
    # Lallemand-Luo rates leave an O(U^2) wall-layer deviation (~2e-7 U here).
    for coll, tol in ((0, 1e-15), (2, 1e-14), (1, 1e-6 * 0.01)):
        cfg = wl.couette_only(8, H, u=0.01, nu=0.2, init_couette=1)
        cfg["collision"] = coll
        s = oracle.Sim(cfg)
        s.step(3000)
        ux, uy, rho = s.fields()
        assert np.abs(ux - exact[:, None]).max() < tol
        assert np.abs(uy).max() < 1e-14 and np.abs(rho - 1).max() < max(tol, 1e-13) * 100


def test_couette_from_rest_converges_to_linear_profile():
    H = 16
    y = np.arange(H) + 0.5
    exact = -0.01 + 0.02 * y / H
    s = oracle.Sim(wl.couette_only(4, H, u=0.01, nu=0.3, init_couette=0))
    s.step(12000)
    ux, _, _ = s.fields()
    assert np.abs(ux - exact[:, None]).max() < 1e-10


def _poiseuille_error(H, nu, coll, g=1e-6, steps=None):
    cfg = wl.couette_only(4, H, u=0.0, nu=nu, init_couette=0)
    cfg.update(gx=g, collision=coll)
    s = oracle.Sim(cfg)
    s.step(steps or int(12 * H * H / nu))
    ux, uy, _ = s.fields()
    y = np.arange(H) + 0.5
    exact = g / (2 * nu) * y * (H - y)
    return np.abs(ux[:, 0] - exact).max() / exact.max(), np.abs(uy).max()


def test_body_force_poiseuille_exact_with_magic_rates():
    # half-way bounce-back puts the no-slip wall exactly at y = 0, H for the
    # magic pairing: the parabola is the exact discrete solution
    for nu in (0.1, 1.0 / 6.0, 0.5):
        err, uy = _poiseuille_error(16, nu, 0)
        assert err < 1e-9 and uy < 1e-14


def test_body_force_poiseuille_second_order_with_other_rates():
    for coll, nu in ((1, 0.1), (2, 0.5)):
        e16, _ = _poiseuille_error(16, nu, coll)
        e32, _ = _poiseuille_error(32, nu, coll)
        assert e16 > 1e-4                      # not exact: wall slip O(1/H^2)
        assert 3.5 < e16 / e32 < 4.5           # second-order convergence


def test_mass_exact_with_beads_forcing_and_moving_walls():
    rng = np.random.default_rng(21)
    cfg = wl.random_fiber(rng, 48, 32, n_beads=5, a=2.0, xi=1.0, gx=2e-6, gy=-1e-6)
    s = oracle.Sim(cfg)
    m0 = s.totals()[0]
    s.step(400)
    assert abs(s.totals()[0] - m0) / m0 < 1e-13


# ------------------------------------------------------------ beads
def _chain(rng, N, NF, a, noise):
    R = np.zeros((N * NF, 2))
    for f in range(NF):
        th = rng.uniform(0, math.pi)
        c = np.array([30.0 + 6.0 * f, 20.0])
        for i in range(N):
            R[f * N + i] = c + (i - (N - 1) / 2) * 2 * a * np.array([math.cos(th), math.sin(th)])
    return R + rng.normal(0, noise, R.shape)


@pytest.mark.parametrize("N,NF", [(2, 1), (3, 1), (4, 1), (5, 1), (9, 1), (7, 2)])
def test_bead_forces_are_minus_energy_gradient(N, NF):
    rng = np.random.default_rng(100 + N)
    a = 2.0
    ks, kb, kev = 3.0, 0.7, 2.5
    R = _chain(rng, N, NF, a, 0.4)
    F = oracle.bead_forces(R, N, NF, a, ks, kb, kev)
    h = 1e-6
    Ffd = np.zeros_like(R)
    for b in range(N * NF):
        for d in range(2):
            Rp = R.copy(); Rp[b, d] += h
            Rm = R.copy(); Rm[b, d] -= h
            Ffd[b, d] = -(oracle.bead_energy(Rp, N, NF, a, ks, kb, kev)
                          - oracle.bead_energy(Rm, N, NF, a, ks, kb, kev)) / (2 * h)
    scale = np.abs(F).max()
    assert np.abs(F - Ffd).max() <= 1e-7 * scale
    # internal forces: no net force, no net torque
    assert np.abs(F.sum(axis=0)).max() <= 1e-13 * scale
    torque = np.sum(R[:, 0] * F[:, 1] - R[:, 1] * F[:, 0])
    assert abs(torque) <= 1e-12 * scale * np.abs(R).max()


def test_bending_alone_is_gradient_and_exercises_every_case():
    # N = 8 uses Eqs. 12a-12e; springs and excluded volume off
    rng = np.random.default_rng(5)
    N, a = 8, 2.0
    R = _chain(rng, N, 1, a, 0.5)
    F = oracle.bead_forces(R, N, 1, a, 0.0, 1.3, 0.0)
    h = 1e-6
    for b in range(N):
        for d in range(2):
            Rp = R.copy(); Rp[b, d] += h
            Rm = R.copy(); Rm[b, d] -= h
            fd = -(oracle.bead_energy(Rp, N, 1, a, 0, 1.3, 0) - oracle.bead_energy(Rm, N, 1, a, 0, 1.3, 0)) / (2 * h)
            assert abs(F[b, d] - fd) <= 1e-7 * np.abs(F).max()


def test_straight_chain_at_rest_length_has_no_force():
    N, a = 10, 4.0
    R = np.array([[10.0 + 8.0 * i, 5.0] for i in range(N)])
    F = oracle.bead_forces(R, N, 1, a, 50.0, 3.0, 2.0)
    assert np.abs(F).max() == 0.0
    # a bend raises the bending energy: -k_b sum t_i.t_{i+1} is minimal straight
    Rb = R.copy(); Rb[5, 1] += 0.5
    assert oracle.bead_energy(Rb, N, 1, a, 0, 3.0, 0) > oracle.bead_energy(R, N, 1, a, 0, 3.0, 0)


def test_excluded_volume_only_for_non_bonded_overlap():
    a = 2.0
    # beads 0 and 2 of one fiber overlap (distance 1 < d = 4): repel
    R = np.array([[0.0, 0.0], [3.0, 2.0], [1.0, 0.0]])
    F = oracle.bead_forces(R, 3, 1, a, 0.0, 0.0, 5.0)
    assert np.allclose(F[0], [-5.0 * 3.0, 0.0]) and np.allclose(F[2], [5.0 * 3.0, 0.0])
    assert np.all(F[1] == 0.0)
    # apart: zero exactly
    R2 = np.array([[0.0, 0.0], [4.0, 0.0], [8.0, 0.0]])
    assert np.abs(oracle.bead_forces(R2, 3, 1, a, 0.0, 0.0, 5.0)).max() == 0.0


# ------------------------------------------------------------ phi, spreading, reduction
def test_phi_profile_values():
    a, xi, rcut, nx = 4.0, 1.0, 12.0, 100.0
    assert math.isclose(oracle.phi(a, xi, rcut, nx, 10.0, 10.0, 10.0, 10.0), 0.5 * (math.tanh(4.0) + 1), rel_tol=1e-15)
    assert math.isclose(oracle.phi(a, xi, rcut, nx, 14.0, 10.0, 10.0, 10.0), 0.5, rel_tol=1e-15)
    assert oracle.phi(a, xi, rcut, nx, 22.0, 10.0, 10.0, 10.0) == 0.0
    v = oracle.phi(a, xi, rcut, nx, 21.9, 10.0, 10.0, 10.0)
    assert 0 < v < 2e-7
    # periodic minimum image in x
    assert oracle.phi(a, xi, rcut, nx, 99.5, 10.0, 1.5, 10.0) == oracle.phi(a, xi, rcut, nx, 3.5, 10.0, 1.5, 10.0)


def test_spread_force_sums_to_bead_forces_and_viscosity_overlay():
    rng = np.random.default_rng(31)
    cfg = wl.random_fiber(rng, 64, 40, n_beads=6, a=2.0, xi=1.0, n_fibers=2, gx=0.0, gy=0.0)
    s = oracle.Sim(cfg)
    R, V, F, S = s.beads()
    fx, fy, nu = s.overlay_fields()
    # Eq. 4: each bead's phi_i F_i / int phi_i integrates back to F_i
    assert abs(fx.sum() - F[:, 0].sum()) < 1e-13 * np.abs(F).max()
    assert abs(fy.sum() - F[:, 1].sum()) < 1e-13 * np.abs(F).max()
    # Eq. 1: fluid viscosity away from beads, ~ r_eta nu_f at bead centres
    nu_f = s.derived()["nu_f"]
    assert nu.min() == nu_f
    j, i = int(R[0, 1]), int(R[0, 0]) % 64
    assert nu[j, i] > 0.5 * cfg["visc_ratio"] * nu_f
    # S_i, the lattice sum of phi, against the continuum integral of Eq. 2:
    # phi = 1 / (1 + exp((r - a)/sigma)) with sigma = xi/2, so
    # int phi dA = 2 pi sigma^2 (-Li2(-exp(a/sigma)))  (cutoff tail < 1e-6)
    from scipy.special import spence
    sig = cfg["xi"] / 2.0
    exact = 2 * math.pi * sig * sig * (-spence(1.0 + math.exp(cfg["a"] / sig)))
    assert np.all(np.abs(S / exact - 1) < 2e-3)


def test_uniform_flow_gives_bead_velocity_exactly():
    # walls moving with the fluid: uniform flow (U, 0) is an exact steady
    # state; with no bead forces V_i must equal U to round-off (Eq. 5)
    U = 0.013
    cfg = wl.couette_only(40, 30, u=0.0, nu=0.2, init_couette=0)
    cfg.update(u_bottom=U, u_top=U, n_beads=4, n_fibers=1, a=2.0, xi=1.0, k_s=0.0, k_b=0.0,
               stiffness_K=0.0, k_ev=0.0, centres=[[20.0, 15.0]], theta0=[0.3])
    s = oracle.Sim(cfg)
    s.set_populations(np.broadcast_to(oracle.feq(1.0, U, 0.0)[:, None, None], (9, 30, 40)).copy())
    R0 = s.beads()[0].copy()
    s.step(6)
    R, V, F, S = s.beads()
    assert np.abs(V - [U, 0.0]).max() < 1e-16
    assert np.abs(R - R0 - 5 * np.array([U, 0.0])).max() < 1e-13


def test_support_integral_nearly_translation_invariant():
    # lattice aliasing of int phi: a reported small number, not exact
    vals = []
    for dx in np.linspace(0, 1, 7):
        cfg = wl.couette_only(64, 48, u=0.01, nu=0.2)
        cfg.update(n_beads=1, n_fibers=1, a=4.0, xi=1.0, centres=[[30.0 + dx, 24.0 + 0.3 * dx]], theta0=[0.0])
        vals.append(oracle.Sim(cfg).beads()[3][0])
    vals = np.array(vals)
    assert (vals.max() - vals.min()) / vals.mean() < 1e-3


def test_derived_parameters_follow_definitions():
    cfg = wl.single_fiber_small()
    d = oracle.Sim(cfg).derived()
    gd = 0.02 / 40
    lc = 8 * 4.0
    assert math.isclose(d["gamma_dot"], gd, rel_tol=1e-15)
    assert math.isclose(d["nu_f"], gd * lc * lc / 1.0, rel_tol=1e-15)           # Re = gd lc^2 / nu
    assert math.isclose(2 * d["k_b"] / (d["nu_f"] * gd * lc * lc), 3.3, rel_tol=1e-14)  # Eq. 18


# ------------------------------------------------------------ sandwich Couette (Sec. 3.1)
def _sandwich_profile(H, r_eta, xi_rel, nu=0.2, U=0.01, steps=None):
    cfg = wl.couette_only(4, H, u=0.0, nu=nu, init_couette=0)
    cfg.update(u_bottom=0.0, u_top=U, visc_ratio=r_eta, xi=xi_rel * H, sandwich_zl=H / 3,
               sandwich_zr=2 * H / 3, threads=min(8, os.cpu_count() or 1))
    s = oracle.Sim(cfg)
    s.step(steps or int(30 * (H / 3) ** 2 / nu) + 2000)
    return s.fields()[0][:, 0], cfg


def _closed_form(H, r_eta, xi, nu, U):
    # steady variable-viscosity Couette flow: constant shear stress, so
    # u(y) = U * int_0^y dy'/nu(y') / int_0^H dy'/nu(y') with nu from Eqs. 1, 14
    from scipy.integrate import quad

    def phi(y):
        if y <= H / 2:
            return 0.5 * (math.tanh((H / 3 - y) / xi) + 1)
        return 0.5 * (math.tanh((y - 2 * H / 3) / xi) + 1)

    inv = lambda y: 1.0 / (nu * (1 + (r_eta - 1) * phi(y)))
    pts = [H / 3, 2 * H / 3]
    total = quad(inv, 0, H, limit=400, points=pts)[0]
    y = np.arange(H) + 0.5
    return np.array([U * quad(inv, 0, v, limit=400, points=[p for p in pts if p < v])[0] / total for v in y])


def test_sandwich_couette_second_order_to_closed_form():
    errs = []
    for H in (30, 60):
        u, cfg = _sandwich_profile(H, 50.0, 0.02)
        errs.append(np.abs(u - _closed_form(H, 50.0, cfg["xi"], 0.2, 0.01)).max() / 0.01)
    assert errs[1] < 3e-3
    assert 3.0 < errs[0] / errs[1] < 4.8        # O(dx^2) at fixed xi / H


def test_sandwich_couette_approaches_eq13_as_interface_thins():
    # Eq. 13: v = 0 below H/3, linear across the fluid layer, V0 above 2H/3.
    # At r_eta = 50 the solids keep O(1/r_eta) of the drop; thinner
    # interfaces (smaller r_xi = xi / H) fit Eq. 13 better (Sec. 3.1).  A
    # larger r_eta alone does not help at a fixed, coarse resolution: the
    # tanh tail times r_eta moves the effective interface ~ (xi/2) ln r_eta
    # into the fluid, which the closed form above accounts for exactly.
    H = 60
    y = np.arange(H) + 0.5
    eq13 = np.clip(0.01 * (y / (H / 3) - 1), 0.0, 0.01)
    dev = []
    for r_xi in (0.04, 0.02, 0.01):
        u, _ = _sandwich_profile(H, 50.0, r_xi)
        dev.append(np.abs(u - eq13).max() / 0.01)
    assert dev[2] < 0.05
    assert dev[0] > dev[1] > dev[2]


# ------------------------------------------------------------ periodic box, driven bead (Sec. 3.2)
def test_external_force_is_gradient_and_periodic_excluded_volume():
    # F_0 on every bead is -grad(-F_0 . R); across the periodic y edge the
    # excluded volume uses the minimum image (energy and force alike)
    rng = np.random.default_rng(9)
    a, ks, kb, kev, ny = 2.0, 3.0, 0.7, 2.5, 30
    R = np.array([[10.0, 1.0], [13.0, 1.5], [16.0, 2.0], [12.0, 28.8], [15.5, 29.5]]) + rng.normal(0, 0.1, (5, 2))
    extra = dict(ny=ny, periodic_y=1, bead_fx=2e-3, bead_fy=-1e-3)
    F = oracle.bead_forces(R, 5, 1, a, ks, kb, kev, **extra)
    h = 1e-6
    for b in range(5):
        for d in range(2):
            Rp = R.copy(); Rp[b, d] += h
            Rm = R.copy(); Rm[b, d] -= h
            fd = -(oracle.bead_energy(Rp, 5, 1, a, ks, kb, kev, **extra)
                   - oracle.bead_energy(Rm, 5, 1, a, ks, kb, kev, **extra)) / (2 * h)
            assert abs(F[b, d] - fd) <= 1e-7 * np.abs(F).max()
    # beads 1 and 4 overlap only through the y edge; without periodicity they do not
    F_walls = oracle.bead_forces(R, 5, 1, a, ks, kb, kev, ny=ny, bead_fx=2e-3, bead_fy=-1e-3)
    assert np.abs(F - F_walls).max() > 1e-3
    # the internal forces still sum to zero: the total is N F_0
    assert np.allclose(F.sum(axis=0), [5 * 2e-3, -5 * 1e-3], rtol=0, atol=1e-14)


def _shear_wave_rate(L, coll, nu=0.1):
    k = 2 * math.pi / L
    s = oracle.Sim(dict(nx=4, ny=L, nu_f=nu, periodic_y=1, init_couette=0, collision=coll,
                        threads=min(4, os.cpu_count() or 1)))
    y = np.arange(L) + 0.5
    fy = np.stack([oracle.feq(1.0, ux, 0.0) for ux in 1e-3 * np.sin(k * y)], axis=1)
    s.set_populations(np.repeat(fy[:, :, None], 4, axis=2).copy())

    def amp():
        return 2.0 / L * float(np.sum(s.fields()[0][:, 0] * np.sin(k * y)))
    s.step(200)
    a1 = amp()
    s.step(2000)
    return math.log(a1 / amp()) / 2000 / (nu * k * k)


@pytest.mark.parametrize("coll", [0, 1, 2])
def test_periodic_shear_wave_decays_at_nu_k2(coll):
    # u_x = U sin(k y) across the periodic y direction decays as exp(-nu k^2 t);
    # the lattice rate converges to nu k^2 at second order in k
    e32, e64 = _shear_wave_rate(32, coll) - 1, _shear_wave_rate(64, coll) - 1
    assert abs(e64) < 2e-3
    assert 3.5 < e32 / e64 < 4.5


def _driven(L, a, xi, r_eta, centre, F0=2e-5, nu=1.0 / 6.0, **kw):
    return oracle.Sim(dict(nx=L, ny=L, nu_f=nu, n_beads=1, n_fibers=1, a=a, xi=xi, visc_ratio=r_eta,
                           periodic_y=1, init_couette=0, bead_fx=F0, gx=-F0 / (L * L), centres=[centre],
                           theta0=[0.0], threads=min(8, os.cpu_count() or 1), **kw))


def test_driven_bead_periodic_translation_invariance_and_momentum_balance():
    # the same bead shifted by whole cells across both periodic edges moves
    # identically; the counter body force keeps the total momentum at zero
    a = _driven(40, 2.0, 0.5, 100.0, [20.3, 20.6])
    b = _driven(40, 2.0, 0.5, 100.0, [20.3 + 17, 20.6 + 19 - 40])  # y = -0.4: across the edge
    a.step(300)
    b.step(300)
    Ra, Va, Fa, Sa = a.beads()
    Rb, Vb, Fb, Sb = b.beads()
    # equal up to the rounding of the shifted coordinates (a wrong wrap
    # would differ at O(1))
    assert abs(Vb[0] - Va[0]).max() <= 1e-10 * abs(Va[0]).max()
    assert abs(Sb[0] - Sa[0]) <= 1e-12 * Sa[0]
    assert abs(b.internal_flow()[0] / a.internal_flow()[0] - 1) < 1e-9
    assert Va[0, 0] > 0 and np.allclose(Fa[0], [2e-5, 0.0], rtol=0, atol=1e-20)
    # the momentum F_0 t put into the bead returns to the fluid exactly (up to
    # rounding of the population sums)
    assert np.abs(a.totals()[1:]).max() < 1e-9 * 2e-5 * 300


def _hasimoto(a, L):
    # drag of a periodic square array of discs in Stokes flow, area fraction c
    c = math.pi * a * a / (L * L)
    return 4 * math.pi / (-0.5 * math.log(c) - 0.738 + c - 0.887 * c * c + 2.039 * c ** 3)


def test_driven_bead_drag_approaches_hasimoto():
    # steady F_0 / (eta V_0) of the FPD disc (a = 2, H = 10 d) against the
    # rigid-disc array: the smooth viscous rim makes the disc hydrodynamically
    # larger than a, by less as the interface thins (r_xi = xi / d)
    ratios = []
    for xi in (0.5, 0.25):
        s = _driven(40, 2.0, xi, 100.0, [20.0, 20.0])
        s.step(int(3 * 40 * 40 / (1.0 / 6.0)))
        V = s.beads()[1][0, 0]
        ratios.append(2e-5 / (V / 6.0) / _hasimoto(2.0, 40))
    assert 1.0 < ratios[1] < ratios[0] < 1.35


def test_internal_flow_vanishes_for_uniform_translation_and_falls_with_viscosity_ratio():
    # a uniformly moving box carries the bead rigidly: eps_v = 0 exactly
    s = oracle.Sim(dict(nx=24, ny=24, nu_f=0.1, n_beads=1, n_fibers=1, a=2.0, xi=0.5, periodic_y=1,
                        init_couette=1, u_bottom=0.01, u_top=0.01, centres=[[12.0, 12.0]], theta0=[0.0]))
    s.step(20)
    assert np.allclose(s.beads()[1][0], [0.01, 0.0], rtol=0, atol=1e-15)
    assert s.internal_flow()[0] < 1e-28
    # Fig. 3d: the residual internal flow of a driven particle falls with r_eta
    ev = []
    for r_eta in (1.0, 10.0, 100.0):
        d = _driven(40, 2.0, 0.25, r_eta, [20.0, 20.0])
        d.step(6000)
        ev.append(d.internal_flow()[0] / d.beads()[1][0, 0] ** 2)
    assert ev[0] > 3 * ev[1] > 9 * ev[2] > 0


# ------------------------------------------------------------ totals (momentum)
def test_total_momentum_grows_by_body_force_each_step_in_periodic_box():
    # Guo forcing adds exactly F to the post-collision momentum of each cell
    # and streaming in a periodic box only moves it: sum_x f c = t g N_cells
    # after t steps from rest, mass N_cells throughout.  A half force counted
    # in the totals, a sign or an x/y mix-up would all break this.
    nx, ny, gx, gy = 24, 18, 3e-6, -1.7e-6
    s = oracle.Sim(dict(wl.couette_only(nx, ny, u=0.0, nu=0.13, init_couette=0), periodic_y=1, gx=gx, gy=gy))
    N = nx * ny
    for t in (0, 1, 5, 40):
        s.step(t - s.nstep)
        m, px, py = s.totals()
        # rounding: each step rounds 9 N populations of size < 1/2, and in a
        # uniform state all cells round alike (coherent), plus the final sum
        floor = (t + 1) * 9 * N * 1.2e-16
        assert abs(m - N) < 1e-12 * N
        assert abs(px - t * gx * N) < floor
        assert abs(py - t * gy * N) < floor
        assert t == 0 or floor < 1e-6 * t * min(abs(gx), abs(gy)) * N  # far below a half-force error


def test_total_momentum_gains_only_the_external_bead_forces():
    # Eq. 4 spreads each bead force with weights phi_i / sum_x phi_i, which sum
    # to one over the lattice, and the springs, bending and excluded volume
    # are internal (they sum to zero): the fluid's momentum grows by the
    # external force on every bead, N_b F_0 per step, and nothing else
    nx = ny = 48
    F0 = np.array([2e-6, -1e-6])
    cfg = dict(wl.couette_only(nx, ny, u=0.0, nu=0.15, init_couette=0), periodic_y=1, n_beads=5, n_fibers=1,
               a=2.0, xi=0.5, stiffness_K=0.0, k_b=0.02, bead_fx=F0[0], bead_fy=F0[1],
               bead_xy=None, centres=[[23.7, 24.2]], theta0=[0.4])
    cfg.pop("bead_xy")
    s = oracle.Sim(cfg)
    R0 = s.beads()[0]
    # a bent start: the chain is not straight, so bending forces act
    R0 = R0 + np.array([[0.0, 0.0], [0.1, -0.2], [0.0, 0.3], [-0.2, 0.1], [0.0, 0.0]])
    s = oracle.Sim(cfg, R0=R0)
    F = s.beads()[2]
    assert np.abs(F - F0).max() > 1e-4   # internal forces are not small
    for t in (1, 7, 30):
        s.step(t - s.nstep)
        m, px, py = s.totals()
        assert abs(m - nx * ny) < 1e-12 * nx * ny
        floor = (t + 1) * 9 * nx * ny * 1.2e-16 + 1e-13 * np.abs(s.beads()[2]).max() * t
        assert abs(px - t * 5 * F0[0]) < floor and abs(py - t * 5 * F0[1]) < floor


def test_total_momentum_of_linear_couette_state_with_unequal_walls():
    # the linear wall profile is the exact discrete steady state: sum_x f c_x
    # = N_x sum_j u(j + 1/2) = N_x N_y (u_bot + u_top) / 2 at every step
    nx, ny, ub, ut = 30, 21, 0.004, 0.012
    cfg = wl.couette_only(nx, ny, u=0.01, nu=0.17, init_couette=1)
    cfg.update(u_bottom=ub, u_top=ut)
    s = oracle.Sim(cfg)
    for t in (0, 3, 50):
        s.step(t - s.nstep)
        m, px, py = s.totals()
        # rounding as in the periodic case, doubled for the bounce-back terms
        floor = (t + 1) * 9 * nx * ny * 2.4e-16
        assert abs(px - nx * ny * (ub + ut) / 2) < floor
        assert abs(py) < floor and abs(m - nx * ny) < 1e-12 * nx * ny


# ------------------------------------------------------------ Eq. 5 weighting
def _phi_moments(a, xi):
    """Continuum moments of the Eq. 2 profile: phi = 1 / (1 + exp((r - a) /
    sigma)), sigma = xi / 2, a Fermi function, whose radial moments are
    int_0^inf r^n phi dr = -sigma^(n+1) n! Li_(n+1)(-exp(a / sigma)).
    Returns int phi dA and the phi-weighted mean of (y - R_y)^2, which is
    (1/2) int phi r^3 dr / int phi r dr."""
    mpmath = pytest.importorskip("mpmath")
    sig = xi / 2.0
    z = -mpmath.e ** (a / sig)
    i1 = -sig ** 2 * mpmath.polylog(2, z)
    i3 = -6 * sig ** 4 * mpmath.polylog(4, z)
    return float(2 * math.pi * i1), float(0.5 * i3 / i1)


def test_bead_velocity_is_phi_weighted_mean_of_a_quadratic_shear_flow():
    # Eq. 5 with u_x = c (y - y0)^2, u_y = 0, no forces (one bead, so no
    # springs; f = 0):  V_x = c ((R_y - y0)^2 + <(y - R_y)^2>_phi),  V_y = 0.
    # The phi-weighted second moment of Eq. 2's profile has the closed form
    # of _phi_moments; at a = 10, xi = 2 the lattice sums differ from the
    # integrals by < 1e-8 (the profile's kink at r = 0 has slope ~e^(-a/sigma)
    # and the edge aliasing is ~exp(-2 pi^2 sigma); the cutoff tail at
    # a + 12 xi is ~1e-10).  Weights phi^2 would give 22.9 instead of 29.09,
    # an unweighted mean over the support ~290.
    nx = ny = 96
    a, xi, c, y0 = 10.0, 2.0, 3e-6, 40.2
    cfg = dict(wl.couette_only(nx, ny, u=0.0, nu=0.1, init_couette=0), periodic_y=1, n_beads=1, n_fibers=1,
               a=a, xi=xi, phi_cut=12.0, k_s=0.0, k_b=0.0, stiffness_K=0.0, k_ev=0.0,
               centres=[[48.3, 47.7]], theta0=[0.0])
    s = oracle.Sim(cfg)
    s.step(1)   # step 0 has no bead advance
    R = s.beads()[0][0].copy()
    y = np.arange(ny) + 0.5
    f = np.stack([oracle.feq(1.0, c * (yy - y0) ** 2, 0.0) for yy in y], axis=1)  # (9, ny)
    s.set_populations(np.repeat(f[:, :, None], nx, axis=2))
    s.step(1)
    R1, V, F, S = s.beads()
    area, m2 = _phi_moments(a, xi)
    assert abs(m2 - 29.0914) < 1e-3
    assert abs(S[0] / area - 1) < 5e-8            # S_i = int phi (Eq. 4's normaliser)
    expect = c * ((R[1] - y0) ** 2 + m2)
    assert abs(V[0, 0] / expect - 1) < 5e-8, (V[0, 0], expect)
    assert abs(V[0, 1]) < 1e-12 * abs(V[0, 0])   # rounding of the u_y sum only
    assert np.allclose(R1[0], R + V[0], rtol=0, atol=1e-15)   # forward Euler, dt = 1
