"""fpd_diag_noalloc (allocation-free diagnostics) against fpd_diag.

fpd_diag_noalloc serves callers that cannot allocate device memory when they
check a running simulation; it keeps its scratch in a fixed device array that
all calls share.  This file is collected last so that a stop-at-first-failure
run has run every other test first; it also passes alone in a fresh process.
Both entry points are called through the C ABI; two calls in a row must each
agree with fpd_diag (the same partial sums, summed in the same order, so the
tolerance used by the other FP64 tests, 1e-12 relative, is met with room).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fpd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14153_gb300 import build, fpd as binding
    build.build()
    return binding


def _check(fpd, sim):
    ref = np.zeros(4)
    fpd.fpd_diag(sim.h, ref)
    for _ in range(2):
        out = np.full(4, np.nan)
        fpd.fpd_diag_noalloc(sim.h, out)
        assert out[3] == ref[3]
        assert np.allclose(out[:3], ref[:3], rtol=1e-12, atol=1e-12 * abs(ref[0])), (out, ref)


def test_noalloc_diag_allocates_nothing_on_a_fresh_handle(fpd):
    # called first on a new handle (before any fpd_diag, which allocates the
    # handle's scratch), the entry point must leave the device's free memory
    # exactly as it was; only then is it compared with fpd_diag
    import torch
    from paper_2212_14153_gb300 import workloads as wl
    # the process's first call loads the library's device module and looks
    # up the array's address: done once here, on another handle
    warm = fpd.Simulation(wl.couette_only(33, 17, precision=1))
    fpd.fpd_diag_noalloc(warm.h, np.zeros(4))
    warm.close()
    sim = fpd.Simulation(wl.two_fiber_large(precision=1))
    sim.step(5)
    sim.sync()
    torch.cuda.synchronize()
    torch.cuda.mem_get_info()
    free0 = torch.cuda.mem_get_info()[0]
    outs = []
    for _ in range(2):
        out = np.full(4, np.nan)
        fpd.fpd_diag_noalloc(sim.h, out)
        outs.append(out)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    ref = np.zeros(4)
    fpd.fpd_diag(sim.h, ref)
    for out in outs:
        assert out[3] == ref[3]
        assert np.allclose(out[:3], ref[:3], rtol=1e-12, atol=1e-12 * abs(ref[0])), (out, ref)
    sim.close()


def test_noalloc_diag_matches_diag_two_calls_in_a_row(fpd):
    from paper_2212_14153_gb300 import workloads as wl
    # a large lattice first (1024 partial blocks), then small ones (few
    # blocks): stale partials of the earlier call must not leak into later ones
    cases = [wl.two_fiber_large(precision=1), wl.single_fiber_small(), wl.couette_only(33, 17, precision=2)]
    for cfg in cases:
        sim = fpd.Simulation(cfg)
        _check(fpd, sim)
        sim.step(7)
        _check(fpd, sim)
        sim.close()


def test_noalloc_diag_reports_nonfinite_state(fpd):
    from paper_2212_14153_gb300 import workloads as wl
    cfg = wl.couette_only(32, 16, u=0.01, nu=0.2)
    cfg["gx"] = 1e300
    sim = fpd.Simulation(cfg)
    sim.step(3)
    out = np.zeros(4)
    with pytest.raises(fpd.FpdError) as e:
        fpd.fpd_diag_noalloc(sim.h, out)
    assert e.value.code == fpd.FPD_ENAN
    sim.close()
