"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 path: relative L2 <= 1e-12 on velocity, populations and bead positions
(the tolerance of the FP64 parity requirement; rounding-order and libm-vs-CUDA
tanh differences are ~1e-16 per step).  Reduced precisions: FP32 math with
FP32 storage of f - w, and FP32 math with FP16 storage of (f - w) 2^s; their
tolerances are derived in the design notes (FP32 unit roundoff 6e-8 times the
step count of the lightly damped modes, FP16 unit roundoff 4.9e-4).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2212_14153_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

THREADS = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14153_gb300 import build
    build.build()


def gpu_sim(cfg, **kw):
    from paper_2212_14153_gb300 import fpd
    return fpd.Simulation(cfg, **kw)


def orc_sim(cfg):
    return oracle.Sim(dict(cfg, threads=THREADS))


def rel_l2(a, b, floor=0.0):
    den = max(np.sqrt(np.sum(b * b)), floor)
    return np.sqrt(np.sum((a - b) ** 2)) / (den if den > 0 else 1.0)


def run_both(cfg, steps):
    g = gpu_sim(cfg)
    o = orc_sim(cfg)
    g.step(steps)
    o.step(steps)
    return g, o


def compare_f64(g, o, tol=1e-12, tol_f=1e-9):
    """Velocity and bead positions/velocities/forces/support sums within
    tol (relative L2).  Floors keep round-off-sized references from turning
    into large relative numbers: the velocity norm is taken as at least that
    of 1e-4 in every component of every cell (1e-4 sqrt(2 ncell)), forces
    against the physical scale below.  The
    population deviations f - w are compared at tol_f: the oracle stores
    plain f (|f| <= 0.45, ulp 5.6e-17), so its own rounding floor relative
    to |f - w| ~ 1e-4 is ~1e-12 per step before any difference in the GPU
    path."""
    ux, uy, rho = g.fields()
    oux, ouy, orho = o.fields()
    ncell = ux.size
    eu = rel_l2(np.stack([ux, uy]), np.stack([oux, ouy]), floor=1e-4 * np.sqrt(2 * ncell))
    w = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    ef = rel_l2(g.populations() - w, o.populations() - w)
    er = abs(rho - orho).max()
    out = dict(u=eu, rho=er)
    if o.nb:
        R, V, F, S = g.beads()
        oR, oV, oF, oS = o.beads()
        out.update(R=rel_l2(R, oR), S=rel_l2(S, oS))
        # V and F are conditioned by R: F ~ (k_s/l0^2)(L - l0) at strains
        # ~1e-4 turns a 1e-16 relative R difference into ~1e-11 in F.  They
        # are compared at 1e-9 against a physical scale: the bending force
        # k_b / l0 plus the spring force at 0.1% strain, and U for V.
        d = o.derived()
        fscale = (d["k_b"] / d["l0"] + 1e-3 * d["k_s"] / d["l0"]) * np.sqrt(2 * o.nb)
        uscale = 1e-2 * np.sqrt(2 * o.nb)
        eV = rel_l2(V, oV, floor=uscale)
        eF = rel_l2(F, oF, floor=fscale)
        assert eV <= 1e-9 and eF <= 1e-9, (eV, eF)
    for k, v in out.items():
        assert v <= tol, (k, v, out, ef)
    assert ef <= tol_f, ("f", ef, out)
    out["f"] = ef
    return out


# ------------------------------------------------------------ fixed points
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_rest_state_is_bit_exact_fixed_point(precision):
    cfg = wl.couette_only(70, 37, u=0.0, nu=0.1, init_couette=0, precision=precision)
    g = gpu_sim(cfg)
    g.step(101)
    f = g.populations()
    assert np.array_equal(f, np.broadcast_to(oracle.feq(1.0, 0.0, 0.0)[:, None, None], f.shape))


@pytest.mark.parametrize("precision,tol", [(0, 1e-16), (1, 2e-8), (2, 2e-5)])
def test_linear_couette_stays_exact(precision, tol):
    H = 37
    cfg = wl.couette_only(45, H, u=0.01, nu=0.2, init_couette=1, precision=precision)
    g = gpu_sim(cfg)
    g.step(2001)
    ux, uy, rho = g.fields()
    exact = -0.01 + 0.02 * (np.arange(H) + 0.5) / H
    assert abs(ux - exact[:, None]).max() < tol
    assert abs(uy).max() < tol


def test_body_force_poiseuille_f64():
    H, nu, gx = 16, 0.1, 1e-6
    cfg = wl.couette_only(33, H, u=0.0, nu=nu, init_couette=0)
    cfg["gx"] = gx
    g = gpu_sim(cfg)
    g.step(int(12 * H * H / nu))
    ux, uy, _ = g.fields()
    y = np.arange(H) + 0.5
    exact = gx / (2 * nu) * y * (H - y)
    assert abs(ux - exact[:, None]).max() / exact.max() < 1e-9


# ------------------------------------------------------------ FP64 parity
@pytest.mark.parametrize("seed,nx,ny,N,NF,a,xi,coll", [
    (1, 70, 37, 5, 1, 2.0, 1.0, 0),     # ragged tiles in x and y
    (2, 96, 48, 6, 2, 2.0, 0.5, 0),     # two fibers, excluded volume across
    (3, 45, 29, 3, 1, 3.0, 1.0, 1),     # N = 3, Lallemand-Luo rates
    (4, 64, 40, 2, 1, 2.5, 1.0, 2),     # N = 2 (no bending), BGK
    (5, 33, 17, 4, 1, 2.0, 1.0, 0),     # support wider than half the lattice
])
def test_fp64_parity_random_cases(seed, nx, ny, N, NF, a, xi, coll):
    rng = np.random.default_rng(seed)
    cfg = wl.random_fiber(rng, nx, ny, n_beads=N, a=a, xi=xi, n_fibers=NF, collision=coll,
                          gx=float(rng.uniform(-1e-6, 1e-6)))
    g, o = run_both(cfg, 301)
    compare_f64(g, o)


def test_fp64_parity_overlapping_beads_excluded_volume():
    # a folded chain: non-bonded beads overlap, so the repulsion is active
    R0 = np.array([[20.0, 15.0], [23.0, 15.0], [23.0, 18.0], [20.5, 17.0], [18.0, 19.0]])
    cfg = wl.couette_only(48, 32, u=0.01, nu=0.5)
    cfg.update(n_beads=5, n_fibers=1, a=2.0, xi=1.0, stiffness_K=0.0, k_b=0.002, k_s=0.05,
               k_ev=0.01, bead_xy=R0)
    g = gpu_sim(cfg)
    o = oracle.Sim(dict(cfg, threads=THREADS), R0=R0)
    assert np.abs(o.beads()[2]).max() > 0
    g.step(200)
    o.step(200)
    assert np.all(np.isfinite(o.beads()[0]))
    compare_f64(g, o)


def test_fp64_parity_pure_fluid_tiny_lattices():
    for nx, ny in [(1, 1), (3, 2), (2, 9), (31, 1)]:
        cfg = wl.couette_only(nx, ny, u=0.01, nu=0.15, init_couette=1)
        cfg["gx"] = 1e-6
        g, o = run_both(cfg, 57)
        compare_f64(g, o)


def test_fp64_parity_small_fiber_config_full_run():
    # 80 x 40, one 8-bead fiber, r_eta = 50, xi = 1, K = 3.3, Re = 1, 10k steps
    cfg = wl.single_fiber_small()
    g, o = run_both(cfg, cfg["steps"])
    res = compare_f64(g, o)
    # the fiber actually moved and rotated, its springs within 2 % strain
    R = g.beads()[0]
    R0 = gpu_sim(cfg).beads()[0]
    assert np.abs(R - R0).max() > 0.05
    L = np.linalg.norm(np.diff(R, axis=0), axis=1)
    assert np.abs(L / (2 * cfg["a"]) - 1).max() < 0.02
    print("config parity", res)


def test_zero_steps_and_step_counter():
    cfg = wl.single_fiber_small()
    g = gpu_sim(cfg)
    g.step(0)
    o = orc_sim(cfg)
    compare_f64(g, o)
    g.step(3)
    assert g.diag()[3] == 3


# ------------------------------------------------------------ population I/O
@pytest.mark.parametrize("parity_steps", [0, 1, 2, 3])
def test_write_read_populations_roundtrip(parity_steps):
    rng = np.random.default_rng(9)
    cfg = wl.couette_only(37, 21, u=0.01, nu=0.2)
    g = gpu_sim(cfg)
    g.step(parity_steps)
    f = oracle.feq(1.0, 0.0, 0.0)[:, None, None] + rng.normal(0, 1e-3, (9, 21, 37))
    g.set_populations(f)
    assert np.array_equal(g.populations(), f)
    # continuing from a written state matches the oracle from the same state
    o = orc_sim(cfg)
    o.set_populations(f)
    g.step(5)
    o.step(5)
    w = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    assert rel_l2(g.populations() - w, o.populations() - w) < 1e-12


def test_uniform_flow_gives_bead_velocity_exactly():
    U = 0.013
    cfg = wl.couette_only(40, 30, u=0.0, nu=0.2, init_couette=0)
    cfg.update(u_bottom=U, u_top=U, n_beads=4, n_fibers=1, a=2.0, xi=1.0, k_s=0.0, k_b=0.0,
               stiffness_K=0.0, k_ev=0.0, centres=[[20.0, 15.0]], theta0=[0.3])
    g = gpu_sim(cfg)
    g.set_populations(np.broadcast_to(oracle.feq(1.0, U, 0.0)[:, None, None], (9, 30, 40)).copy())
    R0 = g.beads()[0].copy()
    g.step(6)
    R, V, F, S = g.beads()
    assert np.abs(V - [U, 0.0]).max() < 1e-16
    assert np.abs(R - R0 - 5 * np.array([U, 0.0])).max() < 1e-13


def test_mass_conserved_on_gpu_f64():
    rng = np.random.default_rng(21)
    cfg = wl.random_fiber(rng, 96, 64, n_beads=6, a=2.0, xi=1.0, gx=2e-6, gy=-1e-6)
    g = gpu_sim(cfg)
    m0 = g.diag()[0]
    g.step(1000)
    assert abs(g.diag()[0] - m0) / m0 < 1e-13


def test_nonfinite_state_reported():
    from paper_2212_14153_gb300 import fpd
    cfg = wl.couette_only(32, 16, u=0.01, nu=0.2)
    cfg["gx"] = 1e300
    g = gpu_sim(cfg)
    g.step(3)
    with pytest.raises(fpd.FpdError) as e:
        g.diag()
    assert e.value.code == fpd.FPD_ENAN


# ------------------------------------------------------------ reduced precision
@pytest.mark.parametrize("precision,tol_u,tol_R", [(1, 1e-4, 1e-6), (2, 2e-2, 1e-3)])
def test_reduced_precision_against_oracle(precision, tol_u, tol_R):
    rng = np.random.default_rng(17)
    cfg = wl.random_fiber(rng, 160, 64, n_beads=8, a=2.0, xi=0.5, precision=precision)
    g = gpu_sim(cfg)
    o = orc_sim(cfg)
    g.step(3000)
    o.step(3000)
    ux, uy, _ = g.fields()
    oux, ouy, _ = o.fields()
    eu = rel_l2(np.stack([ux, uy]), np.stack([oux, ouy]))
    eR = rel_l2(g.beads()[0], o.beads()[0])
    print(f"precision {precision}: rel L2 u {eu:.3e}, R {eR:.3e}")
    assert eu < tol_u and eR < tol_R


# ------------------------------------------------------------ full size
def test_full_size_two_fiber_lattice_f64_and_f32():
    # 4096 x 1024, two 20-bead fibers: the benchmark workload, few steps
    base = wl.two_fiber_large()
    steps = 4
    o = orc_sim(dict(base, precision=0))
    o.step(steps)
    oux, ouy, _ = o.fields()
    oR = o.beads()[0]
    for precision, tol_u, tol_R in [(0, 1e-12, 1e-13), (1, 1e-5, 1e-9), (2, 2e-2, 1e-5)]:
        g = gpu_sim(dict(base, precision=precision))
        g.step(steps)
        ux, uy, _ = g.fields()
        eu = rel_l2(np.stack([ux, uy]), np.stack([oux, ouy]))
        eR = rel_l2(g.beads()[0], oR)
        print(f"full size precision {precision}: rel L2 u {eu:.3e}, R {eR:.3e}")
        assert eu < tol_u and eR < tol_R
        g.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_graph_chunks_equal_direct_steps(precision):
    # one fpd_step(n) call replays captured 32-step graphs; n calls of
    # fpd_step(1) launch every kernel directly: the results must be identical
    rng = np.random.default_rng(77)
    cfg = wl.random_fiber(rng, 70, 37, n_beads=6, a=2.0, xi=1.0, n_fibers=2, precision=precision)
    a = gpu_sim(cfg)
    b = gpu_sim(cfg)
    a.step(101)
    for _ in range(101):
        b.step(1)
    assert np.array_equal(a.populations(), b.populations())
    for x, y in zip(a.beads(), b.beads()):
        assert np.array_equal(x, y)
    a.step(64)           # chunks starting at an odd step
    for _ in range(64):
        b.step(1)
    assert np.array_equal(a.populations(), b.populations())
    # runs shorter than a chunk replay graphs of their own length, captured
    # on first use or beforehand by fpd_prepare: the same bits again
    for n in (2, 3, 5, 20, 31, 33):
        a.prepare(n)
        a.step(n)
        for _ in range(n):
            b.step(1)
    assert a.diag()[3] == b.diag()[3]
    assert np.array_equal(a.populations(), b.populations())
    for x, y in zip(a.beads(), b.beads()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-5), (2, 1e-2)])
def test_sweep_variants_agree(precision, tol, variant):
    # the autotuner's launch shapes (1 cell per thread, 2 cells along x, or
    # a vector of cells along x) compute the same arithmetic; the compiler may
    # contract multiply-adds differently in each instantiation, so they
    # agree to rounding, not bit for bit.  nx = 76: a multiple of the vector
    # width whose last tile is 12 cells wide; ny = 45: ragged rows too
    rng = np.random.default_rng(78)
    cfg = wl.random_fiber(rng, 76, 45, n_beads=6, a=2.0, xi=1.0, n_fibers=2, precision=precision)
    a = gpu_sim(cfg)
    b = gpu_sim(cfg)
    b.set_tuning(variant)
    assert b.tuning() == (variant, 5)
    a.step(77)
    b.step(77)
    w = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    e = rel_l2(b.populations() - w, a.populations() - w)
    print(f"variant {variant} vs 0, precision {precision}: rel L2 of f - w {e:.2e}")
    assert e < tol
    assert rel_l2(b.beads()[0], a.beads()[0]) < tol * 1e-3


@pytest.mark.parametrize("variant", [3, 4])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-4), (2, 1e-2)])
@pytest.mark.parametrize("nx,ny", [
    (160, 150),  # inner blocks of 2, 4 and 8 tiles, ragged top rows
    (203, 282),  # ragged last strip (11 columns), several block rows
])
def test_staged_blocks_against_variant1_and_oracle(precision, tol, variant, nx, ny):
    # variants 3 and 4: blocks of tiles stacked in y whose populations one
    # bulk copy stages in shared memory, the x halo by plain loads; the same
    # cells, collision and stores as variant 1 (FP64 storage runs variant 1).
    # Two fibers that cross inner blocks and block edges; the unmarked tiles
    # of a block go first, the marked ones after the bead phase
    rng = np.random.default_rng(7000 * nx + ny + variant)
    cfg = wl.random_fiber(rng, nx, ny, n_beads=8, a=2.5, xi=1.0, n_fibers=2, precision=precision,
                          gx=float(rng.uniform(-1e-6, 1e-6)))
    a = gpu_sim(cfg)
    a.set_tuning(1)
    b = gpu_sim(cfg)
    b.set_tuning(variant)
    assert b.tuning() == (variant, 5)
    o = orc_sim(cfg)
    for n in (1, 32, 67):  # a direct step, a captured chunk, direct steps
        a.step(n)
        b.step(n)
        o.step(n)
    b.sync()
    assert b.flags() == 0
    w = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    pa, pb = a.populations(), b.populations()
    e = rel_l2(pb - w, pa - w)
    print(f"variant {variant} vs 1, precision {precision}, {nx} x {ny}: rel L2 of f - w {e:.2e}, "
          f"bit-identical {np.array_equal(pa, pb)}")
    assert np.array_equal(pa, pb)  # finish_cells: the same collision and stores as variant 1
    ux, uy, _ = b.fields()
    oux, ouy, _ = o.fields()
    eu = rel_l2(np.stack([ux, uy]), np.stack([oux, ouy]), floor=1e-4 * np.sqrt(2 * ux.size))
    eR = rel_l2(b.beads()[0], o.beads()[0])
    print(f"  vs oracle: rel L2 u {eu:.2e}, R {eR:.2e}")
    assert eu < tol and eR < {0: 1e-12, 1: 1e-6, 2: 1e-4}[precision]


def test_auto_tuning_picks_a_measured_variant_and_caches_it(tmp_path, monkeypatch):
    # Simulation(cfg, tuning="auto") times every launch shape once, keeps the
    # fastest, and a second handle of the same workload reads the cache
    import json
    monkeypatch.setenv("FPD_TUNING_CACHE", str(tmp_path / "tuning.json"))
    rng = np.random.default_rng(79)
    cfg = wl.random_fiber(rng, 96, 48, n_beads=6, a=2.0, xi=1.0, n_fibers=2, precision=1)
    s = gpu_sim(cfg, tuning="auto")
    v, n = s.tuning()
    d = json.load(open(tmp_path / "tuning.json"))
    (entry,) = d.values()
    assert len(entry["ms_per_step"]) == n and entry["variant"] == v
    assert entry["ms_per_step"][v] == min(entry["ms_per_step"])
    assert gpu_sim(cfg, tuning="auto").tuning() == (v, n)
    plain = gpu_sim(cfg)
    assert plain.tuning() == (0, n)
    s.step(40)
    plain.step(40)
    w = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    assert rel_l2(s.populations() - w, plain.populations() - w) < 1e-5


@pytest.mark.parametrize("seed,nx,ny,N,NF,a,xi,coll", [
    (21, 76, 37, 5, 1, 2.0, 1.0, 0),    # last tile 12 cells wide, ragged rows
    (22, 96, 48, 6, 2, 2.0, 0.5, 1),    # two fibers, Lallemand-Luo rates
    (23, 36, 17, 4, 1, 2.0, 1.0, 2),    # support wider than half the lattice, BGK
    (24, 34, 23, 3, 1, 2.5, 1.0, 0),    # FP64 vector width 2: 34 = 32 + 2
])
def test_vector_sweep_fp64_parity(seed, nx, ny, N, NF, a, xi, coll):
    rng = np.random.default_rng(seed)
    cfg = wl.random_fiber(rng, nx, ny, n_beads=N, a=a, xi=xi, n_fibers=NF, collision=coll,
                          gx=float(rng.uniform(-1e-6, 1e-6)))
    g = gpu_sim(cfg)
    g.set_tuning(2)
    o = orc_sim(cfg)
    g.step(301)
    o.step(301)
    compare_f64(g, o)


@pytest.mark.parametrize("seed,nx,ny,N,NF,a,xi,coll", [
    (41, 90, 37, 5, 1, 2.0, 1.0, 0),    # last tile 26 wide: 10 of its threads hold a second cell
    (42, 76, 45, 6, 2, 2.0, 0.5, 1),    # last tile 12 wide: no second cell there
    (43, 20, 17, 3, 1, 2.0, 1.0, 2),    # one tile column: columns 16..19 are second cells, BGK
    (44, 97, 70, 6, 1, 2.0, 1.0, 0),    # inner tiles (precomputed offsets) beside edge tiles
    (45, 7, 9, 3, 1, 1.0, 0.5, 0),      # narrower than the 16-column split
])
def test_two_cells_along_x_fp64_parity(seed, nx, ny, N, NF, a, xi, coll):
    # variant 1: each thread owns two cells of one tile row (x and x + 16 in
    # FP64)
    rng = np.random.default_rng(seed)
    cfg = wl.random_fiber(rng, nx, ny, n_beads=N, a=a, xi=xi, n_fibers=NF, collision=coll,
                          gx=float(rng.uniform(-1e-6, 1e-6)))
    g = gpu_sim(cfg)
    g.set_tuning(1)
    o = orc_sim(cfg)
    g.step(301)
    o.step(301)
    compare_f64(g, o)


@pytest.mark.parametrize("precision,tol", [(1, 1e-4), (2, 1e-2)])
@pytest.mark.parametrize("nx,ny,fiber", [
    (97, 70, True),    # inner tiles: pairs at both strip edges pull across them
    (75, 41, True),    # odd width: the last pair of each row holds one cell
    (130, 28, True),   # five strips, the last two columns wide
    (7, 9, False),     # one strip, narrower than a tile, periodic wrap inside the pairs
])
def test_adjacent_pairs_reduced_precision_against_oracle(precision, tol, nx, ny, fiber):
    # variant 1 in FP32 and FP16 storage: each thread owns two x-adjacent
    # cells, moved with paired accesses, their unforced collision in packed
    # FP32 pairs; against the oracle on ragged lattices
    rng = np.random.default_rng(1000 * nx + ny)
    if fiber:
        cfg = wl.random_fiber(rng, nx, ny, n_beads=4, a=2.0, xi=1.0, precision=precision,
                              gx=float(rng.uniform(-1e-6, 1e-6)))
    else:
        cfg = wl.couette_only(nx, ny, u=0.01, nu=0.15, init_couette=0, precision=precision)
    g = gpu_sim(cfg)
    g.set_tuning(1)
    o = orc_sim(cfg)
    g.step(301)
    o.step(301)
    ux, uy, _ = g.fields()
    oux, ouy, _ = o.fields()
    e = rel_l2(np.stack([ux, uy]), np.stack([oux, ouy]), floor=1e-4 * np.sqrt(2 * ux.size))
    print(f"variant 1, precision {precision}, {nx} x {ny}: rel L2 u {e:.2e}")
    assert e < tol
    if fiber:
        R, oR = g.beads()[0], o.beads()[0]
        assert rel_l2(R, oR) < tol


def test_vector_sweep_tiny_lattices():
    # one vector per row (the lane is both segment ends, the periodic wrap
    # lands in its own vector), single rows, rows of two vectors
    for nx, ny in [(2, 5), (4, 1), (4, 9), (8, 3), (12, 2)]:
        cfg = wl.couette_only(nx, ny, u=0.01, nu=0.15, init_couette=1)
        cfg["gx"] = 1e-6
        cfg["gy"] = -3e-7
        g = gpu_sim(cfg)
        g.set_tuning(2)
        o = orc_sim(cfg)
        g.step(57)
        o.step(57)
        compare_f64(g, o)
        if nx % 4 == 0:
            for p in (1, 2):
                a = gpu_sim(dict(cfg, precision=p))
                b = gpu_sim(dict(cfg, precision=p))
                b.set_tuning(2)
                a.step(57)
                b.step(57)
                assert np.abs(a.populations() - b.populations()).max() < (1e-7 if p == 1 else 1e-5)


def test_vector_variant_falls_back_when_width_does_not_divide_nx():
    # nx = 75: variant 2 runs the one-cell-per-thread sweep, bit for bit
    rng = np.random.default_rng(31)
    cfg = wl.random_fiber(rng, 75, 40, n_beads=5, a=2.0, xi=1.0, precision=1)
    a = gpu_sim(cfg)
    b = gpu_sim(cfg)
    b.set_tuning(2)
    a.step(45)
    b.step(45)
    assert np.array_equal(a.populations(), b.populations())
    for x, y in zip(a.beads(), b.beads()):
        assert np.array_equal(x, y)


def test_sandwich_couette_parity():
    # Sec. 3.1 benchmark: static solid layers (Eq. 14) between walls at 0
    # and V0; FP64 path against the oracle, FP32 against the FP64 path
    H = 45
    cfg = wl.couette_only(12, H, u=0.0, nu=0.2, init_couette=0)
    cfg.update(u_bottom=0.0, u_top=0.01, visc_ratio=50.0, xi=0.9, sandwich_zl=H / 3, sandwich_zr=2 * H / 3)
    g, o = run_both(cfg, 3000)
    compare_f64(g, o)
    g32 = gpu_sim(dict(cfg, precision=1))
    g32.step(3000)
    assert rel_l2(g32.fields()[0], g.fields()[0]) < 1e-4


# ------------------------------------------------------------ periodic box, driven bead (Sec. 3.2)
def driven_cfg(L, a, xi, r_eta, centres, F0=(2e-5, 0.0), n_beads=1, precision=0, **kw):
    nf = len(centres)
    nb = n_beads * nf
    cfg = dict(nx=L, ny=L, u_bottom=0.0, u_top=0.0, nu_f=1.0 / 6.0, re=1.0, visc_ratio=r_eta, xi=xi, a=a,
               n_beads=n_beads, n_fibers=nf, k_s=-1.0, k_b=0.0, stiffness_K=0.0, k_ev=-1.0, phi_cut=8.0,
               collision=0, s_e=1.64, s_eps=1.54, s_q=1.9, init_couette=0, periodic_y=1,
               bead_fx=F0[0], bead_fy=F0[1], gx=-F0[0] * nb / (L * L), gy=-F0[1] * nb / (L * L),
               centres=centres, theta0=[0.0] * nf, precision=precision)
    cfg.update(kw)
    return cfg


@pytest.mark.parametrize("centre", [[20.3, 20.6], [39.2, 39.7], [0.4, 17.0], [13.0, 0.1]])
def test_driven_bead_fp64_parity_across_periodic_edges(centre):
    # F_0 large enough (V ~ 1.5e-2, Re_p ~ 0.4) that the flow stands well
    # above the rounding floor of the oracle's plain-f storage: ulp(f) ~ 6e-17
    # per population and step gives ~1e-13 of |u| here, ~1e-12 at F_0 / 10
    cfg = driven_cfg(40, 2.0, 0.5, 100.0, [centre], F0=(2e-2, -1.3e-2))
    g, o = run_both(cfg, 301)
    compare_f64(g, o)
    eg, eo = g.internal_flow(), o.internal_flow()
    assert abs(eg[0] / eo[0] - 1) < 1e-9, (eg, eo)


def test_periodic_fibers_excluded_volume_across_y_edge_fp64_parity():
    # two 4-bead fibers, one along the bottom edge and one along the top edge
    # one bead diameter apart through the periodic boundary: the excluded
    # volume acts across the edge; each fiber is pushed by F_0
    cfg = driven_cfg(48, 2.0, 0.5, 50.0, [[20.0, 1.5], [20.0, 46.0]], F0=(1e-3, 3e-4), n_beads=4,
                     stiffness_K=0.0, k_b=0.002, k_s=0.05, k_ev=0.01)
    o = orc_sim(cfg)
    g = gpu_sim(cfg)
    # beads 3.5 apart through the edge: fiber 1 is pushed up, fiber 2 down
    F = o.beads()[2]
    assert F[:4, 1].min() > 1e-3 and F[4:, 1].max() < -1e-3
    assert np.abs(g.beads()[2] - F).max() < 1e-12
    R0 = g.beads()[0]
    g.step(250)
    o.step(250)
    compare_f64(g, o)
    assert np.abs(g.beads()[0] - R0).max() > 1e-3


@pytest.mark.parametrize("precision,tol", [(1, 1e-5), (2, 2e-2)])
def test_driven_bead_reduced_precision(precision, tol):
    base = driven_cfg(40, 2.0, 0.5, 100.0, [[39.6, 0.3]], F0=(2e-3, 0.0))
    ref = gpu_sim(base)
    ref.step(2000)
    Vr = ref.beads()[1][0]
    for variant in (0, 1, 2):
        s = gpu_sim(dict(base, precision=precision))
        s.set_tuning(variant)
        s.step(2000)
        V = s.beads()[1][0]
        e = float(np.abs(V - Vr).max() / np.abs(Vr).max())
        print(f"driven bead, precision {precision}, variant {variant}: V rel err {e:.2e}")
        assert e < tol
        assert abs(s.internal_flow()[0] / ref.internal_flow()[0] - 1) < 50 * tol


def test_periodic_shear_wave_on_gpu():
    # u_x = U sin(k y) over the periodic y direction decays as exp(-nu k^2 t)
    L, nu = 64, 0.1
    k = 2 * math.pi / L
    cfg = dict(wl.couette_only(8, L, u=0.0, nu=nu, init_couette=0), periodic_y=1)
    y = np.arange(L) + 0.5
    fy = np.stack([oracle.feq(1.0, ux, 0.0) for ux in 1e-3 * np.sin(k * y)], axis=1)
    f0 = np.repeat(fy[:, :, None], 8, axis=2).copy()
    for p in (0, 1):
        s = gpu_sim(dict(cfg, precision=p))
        s.set_populations(f0)
        s.step(200)
        a1 = 2.0 / L * float(np.sum(s.fields()[0][:, 0] * np.sin(k * y)))
        s.step(2000)
        a2 = 2.0 / L * float(np.sum(s.fields()[0][:, 0] * np.sin(k * y)))
        rate = math.log(a1 / a2) / 2000
        assert abs(rate / (nu * k * k) - 1) < 2e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_early_cold_tiles_give_identical_results(precision, monkeypatch):
    # updating unmarked tiles before the bead phase ends changes only the
    # order of independent work: bit-identical to waiting in every tile
    rng = np.random.default_rng(91)
    cfg = wl.random_fiber(rng, 160, 64, n_beads=6, a=2.0, xi=1.0, n_fibers=2, precision=precision)
    a = gpu_sim(cfg)
    monkeypatch.setenv("FPD_NO_EARLY_COLD", "1")
    b = gpu_sim(cfg)
    monkeypatch.delenv("FPD_NO_EARLY_COLD")
    for s in (a, b):
        s.step(3)
        s.step(64)      # graph chunks
        s.step(5)
    assert np.array_equal(a.populations(), b.populations())
    for x, y in zip(a.beads(), b.beads()):
        assert np.array_equal(x, y)


# ------------------------------------------------------------ checkpoint / resume
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_checkpoint_resume_is_bit_identical(precision, tmp_path):
    rng = np.random.default_rng(55)
    cfg = wl.random_fiber(rng, 70, 37, n_beads=5, a=2.0, xi=1.0, n_fibers=2, precision=precision)
    a = gpu_sim(cfg)
    for split in (41, 42):               # both step parities at the save
        a = gpu_sim(cfg)
        a.step(split)
        path = str(tmp_path / f"ck{split}.fpd")
        a.save(path)
        a.step(70)                       # two graph chunks and a remainder
        b = gpu_sim(cfg)
        b.step(3)                        # a different state, overwritten by the load
        b.load(path)
        assert b.diag()[3] == split
        b.step(70)
        assert np.array_equal(a.populations(), b.populations())
        for x, y in zip(a.beads(), b.beads()):
            assert np.array_equal(x, y)


def test_checkpoint_rejects_other_parameters_and_bad_files(tmp_path):
    from paper_2212_14153_gb300 import fpd
    rng = np.random.default_rng(56)
    cfg = wl.random_fiber(rng, 64, 32, n_beads=4, a=2.0, xi=1.0, precision=1)
    a = gpu_sim(cfg)
    a.step(10)
    path = str(tmp_path / "ck.fpd")
    a.save(path)
    ref = a.populations()
    for other in (dict(cfg, nx=66), dict(cfg, precision=0), dict(cfg, visc_ratio=49.0)):
        c = gpu_sim(other)
        with pytest.raises(fpd.FpdError) as e:
            c.load(path)
        assert e.value.code == fpd.FPD_EINVAL
    raw = open(path, "rb").read()
    bad = {"trunc.fpd": raw[:-7], "junk.fpd": b"not a checkpoint" + raw[16:], "long.fpd": raw + b"x"}
    for name, data in bad.items():
        p = str(tmp_path / name)
        open(p, "wb").write(data)
        with pytest.raises(fpd.FpdError):
            a.load(p)
    with pytest.raises(fpd.FpdError):
        a.load(str(tmp_path / "missing.fpd"))
    # a failed load leaves the handle as it was
    assert np.array_equal(a.populations(), ref)


def test_caller_workspace_gives_identical_results():
    import torch
    from paper_2212_14153_gb300 import fpd
    rng = np.random.default_rng(57)
    cfg = wl.random_fiber(rng, 70, 37, n_beads=5, a=2.0, xi=1.0, precision=1)
    n = fpd.workspace_bytes(cfg)
    ws = torch.empty(n + 512, dtype=torch.uint8, device="cuda")
    a = gpu_sim(cfg)
    b = fpd.Simulation(cfg, workspace=ws[:n])
    a.step(77)
    b.step(77)
    assert np.array_equal(a.populations(), b.populations())
    for x, y in zip(a.beads(), b.beads()):
        assert np.array_equal(x, y)
    b.close()
    ws.fill_(7)                      # still the caller's memory after destroy
    torch.cuda.synchronize()
    for bad in (ws[:n - 256], ws[1:n + 1]):   # too short; misaligned
        with pytest.raises(fpd.FpdError) as e:
            fpd.Simulation(cfg, workspace=bad)
        assert e.value.code == fpd.FPD_EINVAL


@pytest.mark.parametrize("precision", [0, 1])
def test_async_bead_reads_equal_sync_reads(precision):
    # a caller that keeps the next step queued while it consumes the last
    # one's beads (double-buffered pinned reads) sees exactly what the
    # synchronous read returns after the same steps; tickets older than the
    # handle's event ring still wait correctly
    import torch
    rng = np.random.default_rng(91)
    cfg = wl.random_fiber(rng, 96, 40, n_beads=6, a=2.0, xi=1.0, n_fibers=2, precision=precision)
    a, b = gpu_sim(cfg), gpu_sim(cfg)
    nb = a.nb
    bufs = [torch.zeros(7 * nb, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    got, want, prev = [], [], None
    for i in range(20):
        a.step(1)
        t = a.read_beads_async(bufs[i % 2])
        if prev is not None:
            a.wait_read(prev)
            got.append(bufs[(i - 1) % 2].numpy().copy())
        prev = t
        b.step(1)
        R, V, F, S = b.beads()
        want.append(np.concatenate([R[:, 0], R[:, 1], V[:, 0], V[:, 1], F[:, 0], F[:, 1], S]))
    a.wait_read(prev)
    got.append(bufs[19 % 2].numpy().copy())
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    a.wait_read(0)                        # issued 20 reads ago: already complete
    page = np.zeros(7 * nb)               # pageable host memory works too
    a.wait_read(a.read_beads_async(page))
    assert np.array_equal(page, want[-1])
    from paper_2212_14153_gb300 import fpd
    with pytest.raises(fpd.FpdError) as e:
        a.wait_read(10 ** 6)
    assert e.value.code == fpd.FPD_EINVAL


@pytest.mark.parametrize("precision", [0, 1])
def test_bead_export_equals_sync_reads(precision):
    # the bead phase writes every step's finished table into the host ring;
    # taking step n from the ring gives exactly what the synchronous read
    # returns after n steps, for single steps and for graph-replayed chunks
    from paper_2212_14153_gb300 import fpd
    rng = np.random.default_rng(92)
    cfg = wl.random_fiber(rng, 96, 40, n_beads=6, a=2.0, xi=1.0, n_fibers=2, precision=precision)
    a, b = gpu_sim(cfg), gpu_sim(cfg)

    def table(sim):
        R, V, F, S = sim.beads()
        return np.concatenate([R[:, 0], R[:, 1], V[:, 0], V[:, 1], F[:, 0], F[:, 1], S])

    a.export_beads(4)                     # at step 0: the first bead phase finishes step 2
    with pytest.raises(fpd.FpdError) as e:
        a.take_beads(1)
    assert e.value.code == fpd.FPD_EINVAL
    want = {}
    for n in range(1, 25):
        a.step(1)
        b.step(1)
        want[n] = table(b)
        if n >= 3:                        # take the previous step while this one runs
            assert np.array_equal(a.take_beads(n - 1), want[n - 1])
    assert np.array_equal(a.take_beads(24), want[24])
    a.step(64)                            # two captured 32-step chunks
    b.step(64)
    assert np.array_equal(a.take_beads(88), table(b))
    with pytest.raises(fpd.FpdError) as e:  # four slots: step 80 was overwritten
        a.take_beads(80)
    assert e.value.code == fpd.FPD_EBUSY
    with pytest.raises(fpd.FpdError) as e:  # not enqueued
        a.take_beads(89)
    assert e.value.code == fpd.FPD_EINVAL
    a.export_beads(0)
    with pytest.raises(fpd.FpdError) as e:
        a.take_beads(88)
    assert e.value.code == fpd.FPD_EINVAL


def test_bead_export_restarts_after_a_checkpoint_load(tmp_path):
    # a load rewinds the step count; an active export restarts from it and
    # hands over the same tables as an uninterrupted run
    from paper_2212_14153_gb300 import fpd
    rng = np.random.default_rng(93)
    cfg = wl.random_fiber(rng, 80, 40, n_beads=5, a=2.0, xi=1.0, n_fibers=2, precision=1)
    ref = gpu_sim(cfg)
    want = {}
    for n in range(1, 12):
        ref.step(1)
        R, V, F, S = ref.beads()
        want[n] = np.concatenate([R[:, 0], R[:, 1], V[:, 0], V[:, 1], F[:, 0], F[:, 1], S])
    a = gpu_sim(cfg)
    a.step(5)
    path = str(tmp_path / "ck.fpd")
    a.save(path)
    a.export_beads(3)
    a.step(4)
    assert np.array_equal(a.take_beads(9), want[9])
    a.load(path)                          # back at step 5: the export restarts at step 6
    with pytest.raises(fpd.FpdError) as e:
        a.take_beads(9)                   # not enqueued since the load
    assert e.value.code == fpd.FPD_EINVAL
    a.step(6)
    for n in (9, 10, 11):
        assert np.array_equal(a.take_beads(n), want[n])


@pytest.mark.parametrize("variant", [3, 4])
@pytest.mark.parametrize("precision", [1, 2])
def test_staged_blocks_periodic_y_forced_and_sandwich(precision, variant):
    # the staged blocks (variants 3 and 4) on instances whose inner blocks
    # take other paths than an unforced Couette lattice: a driven bead in a
    # box periodic in y with the compensating uniform body force (every cell
    # forced: the moment-form collision on staged populations; blocks at the
    # periodic edges run variant 1's tile code), and the static sandwich
    # layers of Eq. 14 (the viscosity varies across inner blocks without any
    # bead); bit for bit against variant 1 on the same instance
    cases = [driven_cfg(160, 4.0, 1.0, 100.0, [[80.3, 75.6]], F0=(2e-3, 5e-4), precision=precision)]
    H = 150
    sw = wl.couette_only(160, H, u=0.0, nu=0.2, init_couette=0, precision=precision)
    sw.update(u_bottom=0.0, u_top=0.01, visc_ratio=50.0, xi=0.9, sandwich_zl=H / 3, sandwich_zr=2 * H / 3)
    cases.append(sw)
    for cfg in cases:
        a = gpu_sim(cfg)
        a.set_tuning(1)
        b = gpu_sim(cfg)
        b.set_tuning(variant)
        for n in (1, 32, 67):
            a.step(n)
            b.step(n)
        b.sync()
        assert b.flags() == 0
        w = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
        pa, pb = a.populations(), b.populations()
        e = rel_l2(pb - w, pa - w)
        print(f"variant {variant} vs 1, precision {precision}, periodic_y {cfg.get('periodic_y', 0)}, "
              f"sandwich {'sandwich_zl' in cfg}: rel L2 of f - w {e:.2e}, bit-identical {np.array_equal(pa, pb)}")
        assert np.array_equal(pa, pb)
        for x, y in zip(a.beads(), b.beads()):
            assert np.array_equal(x, y)
