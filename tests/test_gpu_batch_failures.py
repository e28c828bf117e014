"""Per-instance failure handling in the batched engine.

An instance that diverges (non-finite state) is found by the batch's
watchdog, reported by fpd_batch_poll as failed (state 3) and taken out of
the running set; the instances beside it run on and stay bit-identical to
their lone runs.  A running instance can be removed (cancelled) at any time
with the same guarantee for the others.
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


def _alone(fpd, cfg, steps):
    s = fpd.Simulation(cfg)
    s.step(steps)
    out = s.populations(), s.beads()
    assert s.flags() == 0
    s.close()
    return out


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)


def _run_all(b, max_steps=700):
    total = 0
    while True:
        d = b.run(max_steps)
        if d == 0:
            return total
        total += d


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_diverged_instance_fails_alone_and_the_others_are_unchanged(fpd, precision):
    rng = np.random.default_rng(500 + precision)
    good = [wl.random_fiber(rng, 70, 37, n_beads=5, a=2.0, xi=1.0, precision=precision),
            wl.random_fiber(rng, 96, 48, n_beads=6, a=2.0, xi=0.5, n_fibers=2, precision=precision)]
    bad = wl.random_fiber(rng, 64, 40, n_beads=4, a=2.0, xi=1.0, precision=precision, gx=1e300)
    steps = 1500     # crosses the watchdog pass at 1024 global steps and ends with one
    b = fpd.Batch(precision, max_slots=4, pool_bytes=64 << 20, max_beads=64)
    s0 = b.add(good[0], steps)
    sb = b.add(bad, steps)
    s1 = b.add(good[1], steps)
    b.run(300)
    # the watchdog pass that ends the run has seen the bad instance
    assert b.flags(sb) & fpd.FPD_FLAG_NONFINITE
    assert b.poll() == [sb] and b.info(sb)["state"] == fpd.SLOT_FAILED
    assert b.info(s0)["state"] == fpd.SLOT_RUNNING and b.flags(s0) == 0
    b.remove(sb)
    _run_all(b)
    assert sorted(b.poll()) == sorted([s0, s1])
    for s, cfg in ((s0, good[0]), (s1, good[1])):
        assert b.info(s)["state"] == fpd.SLOT_FINISHED and b.info(s)["steps_done"] == steps
        assert b.flags(s) == 0
        _same((b.populations(s), b.beads(s)), _alone(fpd, cfg, steps))
    b.close()


def test_instance_diverging_at_its_last_step_is_reported_failed(fpd):
    # the run that brings an instance to its count ends with a watchdog
    # pass, so a diverged instance is never listed as finished
    cfg = wl.couette_only(40, 24, u=0.01, nu=0.2, precision=1)
    cfg["gx"] = 1e300
    b = fpd.Batch(1, max_slots=2, pool_bytes=8 << 20, max_beads=0)
    s = b.add(cfg, 20)
    assert _run_all(b) == 20
    assert b.poll() == [s] and b.info(s)["state"] == fpd.SLOT_FAILED
    b.close()


@pytest.mark.parametrize("precision", [1])
def test_cancelling_a_running_instance_leaves_the_others_unchanged(fpd, precision):
    rng = np.random.default_rng(610)
    cases = [wl.random_fiber(rng, 70, 37, n_beads=5, a=2.0, xi=1.0, precision=precision),
             wl.random_fiber(rng, 80, 40, n_beads=4, a=2.0, xi=0.5, precision=precision),
             wl.couette_only(40, 24, u=0.01, nu=0.2, precision=precision)]
    steps = 400
    b = fpd.Batch(precision, max_slots=4, pool_bytes=64 << 20, max_beads=64)
    slots = [b.add(c, steps) for c in cases]
    b.run(37)
    b.remove(slots[1])          # cancelled while running
    with pytest.raises(fpd.FpdError):
        b.fields(slots[1])
    _run_all(b)
    assert sorted(b.poll()) == sorted([slots[0], slots[2]])
    for i in (0, 2):
        _same((b.populations(slots[i]), b.beads(slots[i])), _alone(fpd, cases[i], steps))
    # the freed slot and its pool room take a new instance, which runs from
    # its own step 0 and matches its lone run too
    s_new = b.add(cases[1], 50)
    _run_all(b)
    _same((b.populations(s_new), b.beads(s_new)), _alone(fpd, cases[1], 50))
    b.close()
