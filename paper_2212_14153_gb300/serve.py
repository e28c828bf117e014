"""Continuous-batching request loop over the batched FPD engine.

Requests (one Couette-fiber simulation each: parameters + step count) arrive
over time.  The loop admits every arrived request for which a slot and pool
room are free (first come, first served, under a device-memory cap), keeps
all admitted instances resident on the device, advances them together in
chunks of time steps, and retires each as soon as it has run its steps
(its bead positions and fields are read back to the host).  Requests that
arrive while others are running join at the next chunk boundary; their work
overlaps on the device with everything already resident, so a request's
time-to-result includes up to one chunk of waiting for admission.

Failures are per request: a request that cannot be admitted even with
nothing resident (its state exceeds the memory cap or the pool, or its
parameters are invalid) is rejected at once, and an instance the batch's
watchdog finds with a non-finite state is retired with an error; the other
requests run on unchanged.

All arithmetic runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import fpd


@dataclass
class Request:
    rid: int
    cfg: dict
    steps: int
    arrival_s: float
    admitted_s: float = -1.0
    done_s: float = -1.0
    slot: int = -1
    result: dict = field(default_factory=dict)
    error: str = ""


def state_bytes(cfg: dict, precision: int) -> int:
    """Device bytes of one instance's populations (two buffers of 9 planes,
    the width padded to whole 32-column strips)."""
    es = {0: 8, 1: 4, 2: 2}[precision]
    align = 32
    pitch = (int(cfg["nx"]) + align - 1) // align * align
    return 2 * 9 * pitch * int(cfg["ny"]) * es


class Server:
    """Continuous batching of FPD requests on one GPU."""

    def __init__(self, precision: int = 1, max_slots: int = 512, cap_bytes: int = 150 << 30,
                 pool_bytes: int | None = None, max_beads: int = 16384, chunk: int = 500,
                 keep_fields: bool = False, stream=None):
        self.precision = precision
        self.cap_bytes = int(cap_bytes)
        self.chunk = int(chunk)
        self.keep_fields = keep_fields
        pool = int(pool_bytes if pool_bytes is not None else cap_bytes)
        self.batch = fpd.Batch(precision, max_slots, min(pool, self.cap_bytes), max_beads, stream)
        self.max_slots = max_slots
        self.resident_bytes = 0

    def close(self):
        self.batch.close()

    def _try_admit(self, req: Request, now: float) -> bool:
        """Admit req if a slot and memory are free; False if it has to wait.
        Raises FpdError for a request the batch refuses outright."""
        need = state_bytes(req.cfg, self.precision)
        if self.resident_bytes + need > self.cap_bytes:
            return False
        try:
            slot = self.batch.add(dict(req.cfg, precision=self.precision), req.steps)
        except fpd.FpdError as e:
            if e.code == fpd.FPD_EBUSY:
                return False
            raise
        req.slot = slot
        req.admitted_s = now
        self.resident_bytes += need
        return True

    @staticmethod
    def _fail(req: Request, now: float, why: str):
        req.error = why
        req.result = {"error": why}
        req.done_s = now

    def _retire(self, req: Request, now: float):
        failed = self.batch.info(req.slot)["state"] == fpd.SLOT_FAILED
        if failed:
            self._fail(req, now, "non-finite state found by the watchdog")
        else:
            R, V, F, S = self.batch.beads(req.slot)
            req.result = {"R": R, "V": V, "F": F}
            if self.keep_fields:
                req.result["fields"] = self.batch.fields(req.slot)
                req.result["populations"] = self.batch.populations(req.slot)
        self.batch.remove(req.slot)
        self.resident_bytes -= state_bytes(req.cfg, self.precision)
        req.done_s = now

    def serve(self, requests: list[Request], clock=time.perf_counter) -> dict:
        """Run all requests (sorted by arrival_s, seconds from start);
        returns latency percentiles and throughput."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        queue: list[Request] = []
        running: dict[int, Request] = {}
        t0 = clock()
        i = 0
        cell_updates = 0.0
        peak = 0  # most requests resident at once
        while i < len(pending) or queue or running:
            now = clock() - t0
            while i < len(pending) and pending[i].arrival_s <= now:
                queue.append(pending[i])
                i += 1
            while queue and len(running) < self.max_slots:
                try:
                    admitted = self._try_admit(queue[0], now)
                except fpd.FpdError as e:
                    self._fail(queue.pop(0), now, f"rejected: {e}")
                    continue
                if not admitted:
                    if not running:
                        # nothing resident: no slot or memory will ever free
                        # up for it, so it cannot run at all
                        r = queue.pop(0)
                        self._fail(r, now, "rejected: does not fit in the empty batch "
                                   f"({state_bytes(r.cfg, self.precision)} state bytes, cap {self.cap_bytes})")
                        continue
                    break
                r = queue.pop(0)
                running[r.slot] = r
            if not running:
                if i < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[i].arrival_s - (clock() - t0))))
                continue
            peak = max(peak, len(running))
            cells = sum(r.cfg["nx"] * r.cfg["ny"] for r in running.values())
            steps = self.batch.run(self.chunk)
            cell_updates += cells * steps
            for slot in self.batch.poll():
                r = running.pop(slot)
                self._retire(r, clock() - t0)
        wall = clock() - t0
        ok = [r for r in requests if not r.error]
        lat = np.array([r.done_s - r.arrival_s for r in ok]) if ok else np.array([np.nan])
        return {
            "requests": len(requests),
            "completed": len(ok),
            "failed": len(requests) - len(ok),
            "wall_s": wall,
            "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()),
            "aggregate_mlups": cell_updates / wall / 1e6,
            "cell_updates": cell_updates,
            "peak_resident": peak,
        }
