"""Driven particle of Sec. 3.2 on the GPU: residual internal flow eps_v and
the drag of the FPD disc in a periodic box (H = 10 d).

Loose physical checks (the paper shows eps_v only as figure curves): eps_v
falls as r_eta grows and as the interface thins (Fig. 3d, e), and the steady
drag approaches Hasimoto's periodic array of rigid discs, from above, as the
interface thins.  Run with -s to see the table.
"""
import pytest

from paper_2212_14153_gb300 import studies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14153_gb300 import build
    build.build()


def test_internal_flow_and_drag_trends():
    pts = ([("r_eta", r, 0.0625, 0.1) for r in (1.0, 10.0, 100.0)]
           + [("r_xi", 100.0, x, 0.1) for x in (0.125, 0.25)])
    out = studies.internal_flow(a=4.0, points=pts)
    rows = out["rows"]
    for r in rows:
        print({k: (round(v, 5) if isinstance(v, float) else v) for k, v in r.items()})
    eps = [r["eps_rel"] for r in rows]
    assert eps[0] > eps[1] > eps[2]            # stiffer particle, less internal flow
    assert eps[2] < eps[3] < eps[4]            # thicker interface, more internal flow
    drag = [r["drag_over_hasimoto"] for r in rows]
    # the viscous rim adds to the disc; less so as the interface thins
    assert 1.0 < drag[2] < 1.25 and drag[2] < drag[3] < drag[4]
    assert max(r["V_drift"] for r in rows) < 1e-3
