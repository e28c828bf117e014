"""Autotuner for the lattice-sweep launch shape.

Each sweep variant (see fpd_set_tuning) is timed with CUDA events on a
scratch instance of the same workload (same parameters, so the same hot
tiles), after warm-up, and the fastest is returned and cached per GPU,
library build, precision and lattice size in a JSON file
($FPD_TUNING_CACHE, default ~/.cache/fpd_gb300/tuning.json): a rebuilt
library (changed kernels) is timed afresh.  Variants compute the same arithmetic
(they differ only in how the compiler contracts multiply-adds, i.e. at the
rounding level), so the choice only affects speed.
"""
from __future__ import annotations

import json
import os

from . import fpd


def _cache_path() -> str:
    return os.environ.get("FPD_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fpd_gb300", "tuning.json"))


def _lib_tag() -> str:
    """Short tag of the built library: its build stamp (a hash of the
    sources, flags and machine), or "unbuilt"."""
    from . import build
    try:
        with open(os.path.join(build.OUT_DIR, "stamp")) as f:
            return f.read().strip()[:12] or "unbuilt"
    except OSError:
        return "unbuilt"


def _key(cfg: dict, gpu: str) -> str:
    return (f"{gpu}|lib{_lib_tag()}|p{cfg.get('precision', 0)}|{cfg['nx']}x{cfg['ny']}"
            f"|nb{cfg.get('n_beads', 0) * cfg.get('n_fibers', 0)}")


def _load() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d: dict) -> None:
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass  # read-only home: tuning still applies to this process


def time_variants(cfg: dict, steps: int = 256, warmup: int = 64, stream=None) -> list[float]:
    """Milliseconds per step of every variant on a scratch instance."""
    import torch
    st = stream or torch.cuda.Stream()
    sim = fpd.Simulation(cfg, stream=st.cuda_stream)
    _, n = sim.tuning()
    out = []
    for v in range(n):
        sim.set_tuning(v)
        sim.step(warmup)
        sim.sync()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        sim.step(steps)
        b.record(st)
        b.synchronize()
        out.append(a.elapsed_time(b) / steps)
    sim.close()
    return out


def tune(cfg: dict, steps: int = 256, warmup: int = 64, use_cache: bool = True) -> int:
    """Fastest sweep variant for this workload (cached)."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _key(cfg, gpu)
    cache = _load() if use_cache else {}
    if key in cache:
        return int(cache[key]["variant"])
    ms = time_variants(cfg, steps, warmup)
    best = int(min(range(len(ms)), key=lambda i: ms[i]))
    cache = _load()
    cache[key] = {"variant": best, "ms_per_step": ms}
    _store(cache)
    return best
