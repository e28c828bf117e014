"""Continuous batching on the GPU: requests admitted while others run give
exactly their alone results."""
import numpy as np
import pytest

from paper_2212_14153_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14153_gb300 import build, fpd, serve
    build.build()
    return fpd, serve


def test_served_results_equal_alone(mods):
    fpd, serve = mods
    rng = np.random.default_rng(12)
    cfgs = [wl.sweep_instance(rng) for _ in range(6)]
    steps = [300, 120, 450, 80, 260, 200]
    reqs = [serve.Request(i, c, n, 0.0) for i, (c, n) in enumerate(zip(cfgs, steps))]
    # two slots: later requests join while earlier ones are running
    srv = serve.Server(precision=1, max_slots=2, cap_bytes=1 << 30, pool_bytes=256 << 20, max_beads=512,
                       chunk=37, keep_fields=True)
    res = srv.serve(reqs)
    srv.close()
    assert res["requests"] == 6
    for r in reqs:
        sim = fpd.Simulation(dict(r.cfg, precision=1))
        sim.step(r.steps)
        assert np.array_equal(r.result["R"], sim.beads()[0])
        assert np.array_equal(r.result["populations"], sim.populations())
        sim.close()
