"""Batched engine (fpd_batch_*): many instances advanced by the same launches.

Every instance must give exactly the numbers it gives alone (the kernels never
mix instances and reduce per instance in a fixed order), whatever its
companions, its slot, its pool offset, or the global step at which it was
admitted.  Compared bit for bit with the single-instance API.
"""
import numpy as np
import pytest

from paper_2212_14153_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fpd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14153_gb300 import build, fpd as binding
    build.build()
    return binding


def _cases(precision):
    rng = np.random.default_rng(40 + precision)
    return [
        wl.random_fiber(rng, 70, 37, n_beads=5, a=2.0, xi=1.0, precision=precision),
        wl.random_fiber(rng, 96, 48, n_beads=6, a=2.0, xi=0.5, n_fibers=2, precision=precision),
        wl.couette_only(40, 24, u=0.01, nu=0.2, precision=precision),
        wl.random_fiber(rng, 33, 17, n_beads=4, a=2.0, xi=1.0, precision=precision, collision=1),
    ]


def _alone(fpd, cfg, steps):
    s = fpd.Simulation(cfg)
    s.step(steps)
    out = s.populations(), s.beads()
    s.close()
    return out


def _same(a, b):
    fa, ba = a
    fb, bb = b
    assert np.array_equal(fa, fb)
    for x, y in zip(ba, bb):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_batch_equals_alone_bit_for_bit(fpd, precision):
    cases = _cases(precision)
    steps = [41, 60, 17, 33]
    b = fpd.Batch(precision, max_slots=8, pool_bytes=64 << 20, max_beads=256)
    slots = [b.add(c, n) for c, n in zip(cases, steps)]
    total = 0
    while True:
        d = b.run(1000)
        if d == 0:
            break
        total += d
    assert total == max(steps)
    done = sorted(b.poll())
    assert done == sorted(slots)
    for c, n, s in zip(cases, steps, slots):
        assert b.info(s)["steps_done"] == n
        _same((b.populations(s), b.beads(s)), _alone(fpd, c, n))
    b.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_fiber_across_the_periodic_edge_and_near_a_wall_batch_equals_alone(fpd, precision):
    # marked tiles that wrap across x = 0 and touch the bottom wall, on a
    # lattice with ragged tiles in x and y: a lone run stages those tiles'
    # bead entries in shared memory, the batch reads them from the table;
    # the same bits either way
    rng = np.random.default_rng(90 + precision)
    cfg = wl.random_fiber(rng, 70, 37, n_beads=5, a=2.0, xi=1.0, n_fibers=2, precision=precision,
                          centres=[[1.5, 8.0], [68.0, 28.5]], theta0=[0.3, 2.6])
    b = fpd.Batch(precision, max_slots=2, pool_bytes=16 << 20, max_beads=64)
    s = b.add(cfg, 57)
    while b.run(1000):
        pass
    assert b.poll() == [s]
    _same((b.populations(s), b.beads(s)), _alone(fpd, cfg, 57))
    b.close()


@pytest.mark.parametrize("precision", [1])
def test_batch_step_and_read_match_run_and_the_split_reads(fpd, precision):
    # fpd_batch_step(n) = fpd_batch_run repeated up to n steps; it stops when
    # every instance has finished; fpd_batch_read = the field and bead reads
    cases = _cases(precision)[:2]
    a = fpd.Batch(precision, max_slots=4, pool_bytes=32 << 20, max_beads=64)
    b = fpd.Batch(precision, max_slots=4, pool_bytes=32 << 20, max_beads=64)
    sa = [a.add(c, n) for c, n in zip(cases, (23, 40))]
    sb = [b.add(c, n) for c, n in zip(cases, (23, 40))]
    a.step(30)
    assert a.info(sa[0])["steps_done"] == 23 and a.info(sa[1])["steps_done"] == 30
    a.step(1000)  # stops at 40: nothing is active any more
    while b.run(1000):
        pass
    for x, y in zip(sa, sb):
        assert a.info(x)["steps_done"] == b.info(y)["steps_done"]
        ux, uy, R = a.read(x)
        fx, fy, _ = b.fields(y)
        assert np.array_equal(ux, fx) and np.array_equal(uy, fy)
        assert np.array_equal(R, b.beads(y)[0])
    with pytest.raises(fpd.FpdError):
        a.step(-1)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_batch_longer_than_the_sms_equals_alone(fpd, precision):
    # a bead list longer than the GPU's SM count runs in narrower bead CTAs
    # than an instance alone; the per-bead sums are taken over the same
    # virtual lanes either way, so every instance still agrees bit for bit
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rng = np.random.default_rng(70 + precision)
    per = 16                                    # beads per instance (2 fibers x 8)
    n_inst = sms // per + 2
    assert n_inst * per > sms >= per
    cases = [wl.random_fiber(rng, 80, 48, n_beads=8, a=2.0, xi=1.0, n_fibers=2, precision=precision)
             for _ in range(n_inst)]
    b = fpd.Batch(precision, max_slots=n_inst, pool_bytes=128 << 20, max_beads=per * n_inst)
    slots = [b.add(c, 12) for c in cases]
    while b.run(1000):
        pass
    for c, s in zip(cases, slots):
        _same((b.populations(s), b.beads(s)), _alone(fpd, c, 12))
    b.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_batch_graph_chunks_equal_alone(fpd, precision):
    # runs long enough that whole 32-step chunks replay captured graphs
    # (started at different mask buffers, across an admission that forces a
    # recapture); every instance still agrees bit for bit
    cases = _cases(precision)
    b = fpd.Batch(precision, max_slots=8, pool_bytes=64 << 20, max_beads=256)
    s0 = b.add(cases[0], 140)
    s1 = b.add(cases[1], 101)
    assert b.run(69) == 69
    s3 = b.add(cases[3], 75)                 # joins at global step 69: recapture
    while b.run(1000):
        pass
    for c, n, s in [(cases[0], 140, s0), (cases[1], 101, s1), (cases[3], 75, s3)]:
        _same((b.populations(s), b.beads(s)), _alone(fpd, c, n))
    b.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-5), (2, 1e-2)])
def test_batch_vector_variant(fpd, precision, tol):
    # variant 2 in a batch: instances whose nx is a multiple of the vector
    # width (96, 40; all four in FP64) run the vector form, the others (70,
    # 33) the column form with that many cells per thread; each agrees with
    # the instance alone to rounding
    cases = _cases(precision)
    steps = [41, 60, 17, 33]
    b = fpd.Batch(precision, max_slots=8, pool_bytes=64 << 20, max_beads=256)
    b.set_tuning(2)
    slots = [b.add(c, n) for c, n in zip(cases, steps)]
    while b.run(1000):
        pass
    w = (np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4))[:, None, None]
    for c, n, s in zip(cases, steps, slots):
        fa, ba = b.populations(s), b.beads(s)
        fb, bb = _alone(fpd, c, n)
        e = np.sqrt(np.sum((fa - fb) ** 2) / np.sum((fb - w) ** 2))
        print(f"batch variant 2 vs alone variant 0, precision {precision}, nx {c['nx']}: "
              f"rel L2 {e:.2e}{' (bit-identical)' if e == 0 else ''}")
        assert e < tol
        if ba[0].size:
            assert np.abs(ba[0] - bb[0]).max() < tol * 1e-2
    b.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-5), (2, 1e-2)])
def test_batch_two_cells_along_x(fpd, precision, tol):
    # variant 1 in a batch (two cells along x per thread, adjacent with paired
    # accesses in the reduced precisions, in-strip pull offsets in inner
    # tiles): each instance
    # agrees with the instance alone to rounding
    cases = _cases(precision) + [wl.couette_only(100, 72, u=0.01, nu=0.2, precision=precision)]
    steps = [41, 60, 17, 33, 25]
    b = fpd.Batch(precision, max_slots=8, pool_bytes=64 << 20, max_beads=256)
    b.set_tuning(1)
    slots = [b.add(c, n) for c, n in zip(cases, steps)]
    while b.run(1000):
        pass
    w = (np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4))[:, None, None]
    for c, n, s in zip(cases, steps, slots):
        fa, ba = b.populations(s), b.beads(s)
        fb, bb = _alone(fpd, c, n)
        e = np.sqrt(np.sum((fa - fb) ** 2) / np.sum((fb - w) ** 2))
        print(f"batch variant 1 vs alone variant 0, precision {precision}, nx {c['nx']}: rel L2 {e:.2e}")
        assert e < tol
        if ba[0].size:
            assert np.abs(ba[0] - bb[0]).max() < tol * 1e-2
    b.close()


def test_staggered_admission_and_slot_reuse(fpd):
    cases = _cases(1)
    b = fpd.Batch(1, max_slots=3, pool_bytes=64 << 20, max_beads=128)
    s0 = b.add(cases[0], 50)
    assert b.run(7) == 7
    s1 = b.add(cases[1], 30)                 # joins at global step 7 (odd)
    assert b.run(10) == 10
    s2 = b.add(cases[3], 25)                 # joins at global step 17
    while b.run(1000):
        pass
    assert sorted(b.poll()) == sorted([s0, s1, s2])
    for c, n, s in [(cases[0], 50, s0), (cases[1], 30, s1), (cases[3], 25, s2)]:
        _same((b.populations(s), b.beads(s)), _alone(fpd, c, n))
    # free a slot and reuse it (and its pool room) for another instance
    b.remove(s1)
    s3 = b.add(cases[2], 12)
    assert s3 == s1
    while b.run(1000):
        pass
    _same((b.populations(s3), b.beads(s3)), _alone(fpd, cases[2], 12))
    b.close()


def test_admission_limits(fpd):
    cfg = wl.couette_only(64, 64, precision=1)
    pool = 2 * 9 * 64 * 64 * 4 * 2 + 4096      # room for two such lattices (two buffers each)
    b = fpd.Batch(1, max_slots=4, pool_bytes=pool, max_beads=8)
    b.add(cfg, 5)
    b.add(cfg, 5)
    with pytest.raises(fpd.FpdError) as e:
        b.add(cfg, 5)
    assert e.value.code == fpd.FPD_EBUSY
    rng = np.random.default_rng(3)
    big = wl.random_fiber(rng, 32, 16, n_beads=9, a=1.5, xi=0.5, precision=1)
    with pytest.raises(fpd.FpdError):          # 9 beads > room for 8
        b.add(big, 5)
    with pytest.raises(fpd.FpdError) as e:     # precision mismatch
        b.add(wl.couette_only(16, 16, precision=0), 5)
    assert e.value.code == fpd.FPD_EINVAL
    st = b.stats()
    assert st["running"] == 2 and st["pool_used"] > 0
    b.close()


def test_batched_sweep_instances_run_and_conserve_mass(fpd):
    inst = wl.batched_sweep(n=24, seed=11)
    b = fpd.Batch(1, max_slots=32, pool_bytes=1 << 30, max_beads=1024)
    slots = [b.add(c, 200) for c in inst]
    while b.run(64):
        pass
    for c, s in zip(inst, slots):
        f = b.populations(s)
        assert np.all(np.isfinite(f))
        m = f.sum()
        assert abs(m - c["nx"] * c["ny"]) / (c["nx"] * c["ny"]) < 1e-5
        R = b.beads(s)[0]
        assert np.all(np.isfinite(R))
    b.close()


def test_periodic_driven_instances_in_a_batch(fpd):
    # periodic boxes with a driven bead next to walled Couette cells: each
    # instance gives exactly what it gives alone
    cases = [
        dict(nx=40, ny=40, u_bottom=0.0, u_top=0.0, nu_f=1.0 / 6.0, visc_ratio=100.0, xi=0.5, a=2.0,
             n_beads=1, n_fibers=1, init_couette=0, periodic_y=1, bead_fx=2e-5, gx=-2e-5 / 1600,
             centres=[[39.5, 0.2]], theta0=[0.0], precision=p)
        for p in (0, 1)
    ]
    for p in (0, 1):
        mixed = [cases[p], _cases(p)[0]]
        b = fpd.Batch(p, max_slots=4, pool_bytes=32 << 20, max_beads=64)
        slots = [b.add(c, 120) for c in mixed]
        while b.run(1000):
            pass
        for c, s in zip(mixed, slots):
            _same((b.populations(s), b.beads(s)), _alone(fpd, c, 120))
        b.close()
