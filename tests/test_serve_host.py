"""Host-side scheduling of the continuous-batching loop (no GPU): a fake
batch stands in for the device engine and advances instances by counting."""
import numpy as np
import pytest

from paper_2212_14153_gb300 import fpd, serve


class FakeBatch:
    def __init__(self, precision, max_slots, pool_bytes, max_beads, stream=None):
        self.max_slots, self.pool, self.used = max_slots, pool_bytes, 0
        self.slots = {}
        self.log = []
        self.fail_at = set()  # step counts whose instances the fake reports as failed

    def add(self, cfg, n):
        need = serve.state_bytes(cfg, 1)
        free = [s for s in range(self.max_slots) if s not in self.slots]
        if not free or self.used + need > self.pool:
            raise fpd.FpdError(fpd.FPD_EBUSY, "full")
        s = free[0]
        self.slots[s] = [0, n, need]
        self.used += need
        self.log.append(("add", cfg["rid"], s))
        return s

    def run(self, k):
        act = [v for v in self.slots.values() if v[0] < v[1]]
        if not act:
            return 0
        k = min(k, min(v[1] - v[0] for v in act))
        for v in act:
            v[0] += k
        return k

    def poll(self):
        out = [s for s, v in self.slots.items() if v[0] >= v[1] and len(v) == 3]
        for s in out:
            self.slots[s].append("reported")
        return out

    def info(self, slot):
        v = self.slots[slot]
        failed = v[1] in self.fail_at
        return dict(state=fpd.SLOT_FAILED if failed else fpd.SLOT_FINISHED)

    def beads(self, slot):
        return np.zeros((1, 2)), np.zeros((1, 2)), np.zeros((1, 2)), np.zeros(1)

    def remove(self, slot):
        self.used -= self.slots[slot][2]
        del self.slots[slot]

    def close(self):
        pass


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(fpd, "Batch", FakeBatch)


def _req(i, nx, ny, steps, t):
    cfg = dict(nx=nx, ny=ny, rid=i)
    return serve.Request(i, cfg, steps, t)


def test_all_requests_complete_with_positive_latency(fake):
    srv = serve.Server(max_slots=3, cap_bytes=1 << 30, chunk=100)
    reqs = [_req(i, 64, 32, 150 + 50 * i, 0.002 * i) for i in range(10)]
    res = srv.serve(reqs, clock=FakeClock())
    assert res["requests"] == 10
    for r in reqs:
        assert r.done_s >= r.admitted_s >= r.arrival_s >= 0
    assert res["p99_s"] >= res["p50_s"] > 0
    assert res["aggregate_mlups"] > 0


def test_slot_limit_and_fifo_admission(fake):
    srv = serve.Server(max_slots=2, cap_bytes=1 << 30, chunk=50)
    reqs = [_req(i, 32, 32, 100, 0.0) for i in range(5)]
    res = srv.serve(reqs, clock=FakeClock())
    assert res["peak_resident"] == 2
    order = [rid for kind, rid, s in srv.batch.log if kind == "add"]
    assert order == [0, 1, 2, 3, 4]                     # first come, first served
    adm = sorted(reqs, key=lambda r: r.admitted_s)
    assert adm[2].admitted_s >= min(adm[0].done_s, adm[1].done_s)  # waited for a slot


def test_memory_cap_limits_residency(fake):
    one = serve.state_bytes(dict(nx=128, ny=64), 1)
    srv = serve.Server(max_slots=16, cap_bytes=2 * one + 10, chunk=50)
    reqs = [_req(i, 128, 64, 100, 0.0) for i in range(4)]
    res = srv.serve(reqs, clock=FakeClock())
    assert res["peak_resident"] == 2 and res["completed"] == 4
    # at most two resident at any time: the third admission follows a retirement
    adm = sorted(reqs, key=lambda r: r.admitted_s)
    assert adm[2].admitted_s >= min(r.done_s for r in adm[:2])
    assert srv.resident_bytes == 0


def test_state_bytes_pads_width_to_whole_strips():
    # two buffers of 9 planes, the width padded to 32-column strips
    assert serve.state_bytes(dict(nx=80, ny=40), 1) == 2 * 9 * 96 * 40 * 4
    assert serve.state_bytes(dict(nx=80, ny=40), 2) == 2 * 9 * 96 * 40 * 2
    assert serve.state_bytes(dict(nx=64, ny=10), 0) == 2 * 9 * 64 * 10 * 8
    assert serve.state_bytes(dict(nx=65, ny=10), 0) == 2 * 9 * 96 * 10 * 8


def test_request_larger_than_the_cap_is_rejected_not_spun_on(fake):
    # a request whose state alone exceeds the memory cap can never be
    # admitted; with nothing resident the loop must reject it instead of
    # waiting forever, and serve the others
    one = serve.state_bytes(dict(nx=64, ny=32), 1)
    srv = serve.Server(max_slots=4, cap_bytes=4 * one, chunk=50)
    big = _req(0, 4096, 4096, 100, 0.0)
    reqs = [big] + [_req(i, 64, 32, 100, 0.0) for i in range(1, 4)]
    res = srv.serve(reqs, clock=FakeClock())
    assert big.error.startswith("rejected") and big.slot == -1
    assert res["failed"] == 1 and res["completed"] == 3
    assert all(not r.error and r.result for r in reqs[1:])
    assert srv.resident_bytes == 0


def test_request_the_batch_refuses_outright_is_rejected(fake, monkeypatch):
    plain_add = FakeBatch.add

    def add(self, cfg, n):
        if cfg["rid"] == 1:
            raise fpd.FpdError(fpd.FPD_EINVAL, "bad parameters")
        return plain_add(self, cfg, n)
    monkeypatch.setattr(FakeBatch, "add", add)
    srv = serve.Server(max_slots=4, cap_bytes=1 << 30, chunk=50)
    reqs = [_req(i, 64, 32, 100, 0.0) for i in range(3)]
    res = srv.serve(reqs, clock=FakeClock())
    assert reqs[1].error.startswith("rejected") and res["completed"] == 2


def test_failed_instance_is_retired_with_an_error_and_others_continue(fake):
    srv = serve.Server(max_slots=4, cap_bytes=1 << 30, chunk=50)
    srv.batch.fail_at = {150}     # the fake reports the 150-step request failed
    reqs = [_req(0, 64, 32, 100, 0.0), _req(1, 64, 32, 150, 0.0), _req(2, 64, 32, 200, 0.0)]
    res = srv.serve(reqs, clock=FakeClock())
    assert reqs[1].error and "non-finite" in reqs[1].result["error"]
    assert not reqs[0].error and not reqs[2].error and "R" in reqs[2].result
    assert res["completed"] == 2 and res["failed"] == 1
    assert srv.resident_bytes == 0 and not srv.batch.slots
