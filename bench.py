"""Benchmark of the FPD-MRT time step (MLUPS and fraction of the HBM roofline).

Workload: the two-fiber lattice, 4096 x 1024 cells, two 20-bead fibers
(a = 4, xi = 1), r_eta = 50, K = 0.33, Re = 5, walls -/+0.01, seeded angles;
synthetic, as the paper prints no input data.  One "step" is one full time
step of the method (bead phase + fused collide/stream/bounce-back sweep).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision 0|1|2]
    python bench.py --impl reference      # the FP64 CPU oracle on host cores
    python bench.py --workload sweep --steps 500 --warmup 5   # batched vs plain loop
    python bench.py --workload serve --instances 200          # continuous batching

Prints one JSON line (rank 0).  For N > 1 (torchrun) every rank runs its own
instance of the workload (independent sweep points: weak scaling, no data
exchange) and the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PRECISION_NAMES = {0: "f64", 1: "f32", 2: "f32 (f16 storage)"}
STORE_BYTES = {0: 8, 1: 4, 2: 2}
L2_BYTES = 129 * 2 ** 20


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("fpd_lattice.cu", "fpd_device.cuh"):
        with open(os.path.join(ROOT, "paper_2212_14153_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, precision: int, variant: int):
    """DRAM bytes per launch of the lattice kernel (the given sweep variant)
    from the committed ncu summary, if it was taken on the current kernel
    source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[f"{workload}:{precision}:v{variant}"]
        if e.get("kernel_hash") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_launch_full"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        if shutil.which("nvidia-smi"):
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def l2_note(state_bytes: int) -> str:
    mib = state_bytes / 2 ** 20
    if state_bytes > L2_BYTES:
        return f"state {mib:.0f} MiB > 129 MiB L2: every step streams from HBM, no flush needed"
    return f"state {mib:.0f} MiB fits in the 129 MiB L2: L2-resident, not an HBM measurement"


def pick_variant(args, cfg):
    """Sweep launch shape: fixed by --variant, or timed by the autotuner."""
    if args.variant != "auto":
        return int(args.variant), None
    from paper_2212_14153_gb300 import autotune
    ms = autotune.time_variants(cfg, steps=128, warmup=32)
    return int(min(range(len(ms)), key=lambda i: ms[i])), [round(m, 5) for m in ms]


# ------------------------------------------------------------------ GPU arm
def gpu_state(fpd, cfg, precision, variant, steps, stream):
    """(u_x, u_y, R) after `steps` steps of cfg at this precision and sweep
    variant, run as the timed region runs it (graph chunks)."""
    s = fpd.Simulation(dict(cfg, precision=precision), stream=stream.cuda_stream)
    s.set_tuning(variant)
    s.step(steps)
    ux, uy, _ = s.fields()
    R = s.beads()[0]
    s.close()
    return ux, uy, R


def accuracy_vs_fp64(fpd, cfg, precision, variant, steps, stream):
    """The timed configuration against FP64 storage (the path pinned to the
    oracle at 1e-12) after a short run."""
    ux64, uy64, R64 = gpu_state(fpd, cfg, 0, variant, steps, stream)
    ux, uy, R = gpu_state(fpd, cfg, precision, variant, steps, stream)
    u64 = np.concatenate([ux64.ravel(), uy64.ravel()])
    u = np.concatenate([ux.ravel(), uy.ravel()])
    return {"vs": "FP64 storage on this GPU (pinned to the oracle at 1e-12)", "steps": steps,
            "sweep_variant": variant, "u_rel_l2": float(np.linalg.norm(u - u64) / np.linalg.norm(u64)),
            "bead_max_dR": float(np.abs(R - R64).max())}


def batched_leg(fpd, workloads, stream, n_inst: int, steps: int, warm: int = 8) -> dict:
    """The batched sweep (n_inst instances drawn as the shape-diagram sweep,
    FP32) against the plain loop that runs the same instances one at a time
    with the same kernels, and the bit-identity of two instances with their
    lone runs."""
    import torch
    from paper_2212_14153_gb300 import serve
    inst = workloads.batched_sweep(n=n_inst, seed=4, precision=1)
    cells = [c["nx"] * c["ny"] for c in inst]
    pool = sum(serve.state_bytes(c, 1) + 4096 for c in inst)
    nbeads = sum(c["n_beads"] * c["n_fibers"] for c in inst)
    b = fpd.Batch(1, len(inst), pool, nbeads, stream=stream.cuda_stream)
    slots = [b.add(c, warm + steps) for c in inst]
    b.run(warm)
    b.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    done = 0
    while done < steps:
        d = b.run(steps - done)
        if d == 0:
            break
        done += d
    e1.record(stream)
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) * 1e-3
    b.poll()
    check = {}
    for i in (0, len(inst) // 2):
        fb, Rb = b.populations(slots[i]), b.beads(slots[i])[0]
        s1 = fpd.Simulation(inst[i], stream=stream.cuda_stream)
        s1.step(warm + steps)
        check[i] = bool(np.array_equal(fb, s1.populations()) and np.array_equal(Rb, s1.beads()[0]))
        s1.close()
    b.close()
    t_plain = 0.0
    for c in inst:
        s1 = fpd.Simulation(c, stream=stream.cuda_stream)
        s1.step(warm)
        s1.sync()
        e0.record(stream)
        s1.step(steps)
        e1.record(stream)
        e1.synchronize()
        t_plain += e0.elapsed_time(e1) * 1e-3
        s1.close()
    batched = sum(cells) * steps / t_batch / 1e6
    plain = sum(cells) * steps / t_plain / 1e6
    return {"workload": "batched_sweep", "instances": len(inst), "cells": sum(cells), "beads": nbeads,
            "steps": steps, "storage": "f32", "sweep_variant": 0, "value": round(batched, 1), "unit": "MLUPS",
            "plain_loop": round(plain, 1), "speedup": round(batched / plain, 2),
            "ms_per_step": t_batch * 1e3 / steps,
            "roofline_frac": round(72 * sum(cells) * steps / t_batch / 1e9 / measured_peaks()["hbm_gbs"], 4),
            "bit_identical_to_alone": check,
            "accuracy": "every instance bit-identical to its lone run (checked here on two)"}


def fp16_leg(args, fpd, workloads, stream, steps: int = 2000) -> dict:
    """The two-fiber step with FP16 storage (FP32 math): whole-step and
    sweep-kernel rooflines at 36 B per cell update, and accuracy against FP64
    storage in the same launch shape."""
    import torch
    cfg = workloads.two_fiber_large(seed=3, precision=2)
    cells = cfg["nx"] * cfg["ny"]
    variant, variant_ms = pick_variant(args, cfg)
    sim = fpd.Simulation(cfg, stream=stream.cuda_stream)
    sim.set_tuning(variant)
    sim.step(max(args.warmup, 32))
    sim.prepare(steps)
    sim.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    sim.set_profiling(True)
    sim.step(steps)
    kt = sim.kernel_times()
    sim.set_profiling(False)
    sim.close()
    peak = measured_peaks()["hbm_gbs"]
    lat_ms = kt["lattice_ms"] / max(kt["lattice_launches"], 1)
    return {"workload": cfg["name"], "storage": "f16x2^s", "sweep_variant": variant, "variant_ms_per_step": variant_ms,
            "steps": steps, "ms_per_step": ms, "value": round(cells / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
            "step_frac": round(36 * cells / (ms * 1e-3) / 1e9 / peak, 4),
            "kernel_ms": lat_ms, "kernel_frac": round(36 * cells / (lat_ms * 1e-3) / 1e9 / peak, 4),
            "accuracy": accuracy_vs_fp64(fpd, cfg, 2, variant, args.accuracy_steps, stream)}


def run_gpu(args, rank: int, world: int):
    import torch
    from paper_2212_14153_gb300 import build, fpd, replicas, workloads

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    build.build()
    cfg = workloads.two_fiber_large(seed=3 + rank, precision=args.precision)
    cells = cfg["nx"] * cfg["ny"]
    stream = torch.cuda.Stream()
    variant, variant_ms = pick_variant(args, cfg)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- device-resident throughput (value): consecutive launches overlap
    # (programmatic dependent launch), so no per-kernel events in this region
    sim = fpd.Simulation(cfg, stream=stream.cuda_stream)
    sim.set_tuning(variant)
    sim.step(args.warmup)
    # the step graphs the timed call replays are captured before timing
    sim.prepare(args.steps)
    sim.sync()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if rank == 0 else None
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    sim.step(args.steps)
    end.record(stream)
    end.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = start.elapsed_time(end)
    # ---- live per-kernel durations: a second timed region of the same
    # length with CUDA events around every launch on the library's stream
    sim.set_profiling(True)
    sim.step(args.steps)
    kt = sim.kernel_times()
    sim.set_profiling(False)
    diag = sim.diag()
    sim.close()
    # whole job: every rank's cell updates over the slowest rank's time
    mlups = replicas.job_rate(cells * args.steps, ms * 1e-3) / 1e6
    ms = replicas.max_over_ranks(ms)

    # ---- end to end through the public API with host buffers: the final
    # fields go into page-locked host buffers allocated beforehand (as a
    # caller reading results repeatedly would keep them), every step's bead
    # table into the handle's page-locked ring
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    field_bufs = tuple(torch.empty((cfg["ny"], cfg["nx"]), dtype=torch.float64, pin_memory=True).numpy()
                       for _ in range(3))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = fpd.Simulation(cfg, stream=stream.cuda_stream)
    sim.set_tuning(variant)
    nb = sim.nb
    # every step's bead table comes back to the host: the bead phase writes it
    # into a host ring itself (no copy between the kernels of the step
    # chain), and the host takes step n while step n + 1 runs
    sim.export_beads(4)
    dst = np.empty(7 * max(nb, 1))
    taken = 0.0
    t_loop0 = time.perf_counter()
    for i in range(e2e_steps):
        sim.step(1)
        n = i + 1
        if n == 1:
            R, V, F, S = sim.beads()          # step 1 has no bead phase: the initial table
            taken += R[0, 0] if nb else 0.0
        elif n >= 3:
            sim.take_beads(n - 1, dst)
            taken += dst[0]
    if e2e_steps >= 2:
        sim.take_beads(e2e_steps, dst)
        taken += dst[0]
    t_loop = time.perf_counter() - t_loop0
    ux, uy, rho = sim.fields(out=field_bufs)
    sim.close()
    e2e_s = time.perf_counter() - t0
    e2e_mlups = replicas.job_rate(cells * e2e_steps, e2e_s) / 1e6
    h2d_total = 200 + 8 * 2 * cfg["n_fibers"] * 2 + 8 * 2 * nb  # params, centres/angles, bead table
    d2h_step = 8 * 7 * nb                                        # R, V, F, S every step
    d2h_total = d2h_step * e2e_steps + 3 * 8 * cells             # + final u_x, u_y, rho

    # accuracy beside the throughput: the same workload in FP64 storage (the
    # path the parity tests pin to the oracle at 1e-12) against this
    # precision, after a short run
    accuracy = None
    if rank == 0 and args.precision != 0 and args.accuracy_steps > 0:
        accuracy = accuracy_vs_fp64(fpd, cfg, args.precision, variant, args.accuracy_steps, stream)

    # batched sweep against the plain loop, and the FP16-storage step, on
    # the same GPU (fixed sizes, independent of --steps)
    batched = fp16 = None
    if rank == 0 and not args.no_extras:
        batched = batched_leg(fpd, workloads, stream, args.batched_instances, args.batched_steps)
        if args.precision != 2:
            fp16 = fp16_leg(args, fpd, workloads, stream)

    if rank == 0:
        peaks = measured_peaks()
        bpc = 18 * STORE_BYTES[args.precision]
        lat_ms = kt["lattice_ms"] / max(kt["lattice_launches"], 1)
        achieved = bpc * cells / (lat_ms * 1e-3) / 1e9
        step_gbs = bpc * cells * args.steps / (ms * 1e-3) / 1e9
        traffic = ncu_traffic(cfg["name"], args.precision, variant)
        gpu_launches = kt["lattice_launches"] + kt["bead_launches"]  # per timed region
        line = {
            "metric": "MLUPS (million lattice-cell updates per second) of the FPD-MRT step",
            "value": round(mlups, 1),
            "unit": "MLUPS",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": {0: "f64", 1: "f32", 2: "f32"}[args.precision],
            "data": "synthetic",
            "config": {
                "workload": cfg["name"], "nx": cfg["nx"], "ny": cfg["ny"], "fibers": cfg["n_fibers"],
                "beads_per_fiber": cfg["n_beads"], "storage": {0: "f64", 1: "f32", 2: "f16x2^s"}[args.precision],
                "bytes_per_cell_update": bpc, "per_gpu": "one independent instance",
                "l2": l2_note(bpc * cells), "sweep_variant": variant, "variant_ms_per_step": variant_ms,
                "parallelism": f"replicas x{world}",
            },
            "roofline": {
                "bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "kernel": "k_lattice", "kernel_ms": lat_ms, "peak_source": peaks["source"],
                "bead_kernel_ms": kt["bead_ms"] / max(kt["bead_launches"], 1),
                # the whole step (bead phase included) as a fraction of the
                # roofline: bytes per cell update x cell updates per second
                "step_achieved": round(step_gbs, 1), "step_frac": round(step_gbs / peaks["hbm_gbs"], 4),
            },
            "gpu_launches": gpu_launches,
            "e2e": {"value": round(e2e_mlups, 1), "unit": "MLUPS", "h2d_bytes_per_step": h2d_total / e2e_steps,
                    "d2h_bytes_per_step": d2h_total / e2e_steps, "steps": e2e_steps,
                    # the step loop alone (per step: fpd_step(1) and the host
                    # taking that step's bead table), without create, the
                    # final field read and destroy, which a run of e2e_steps
                    # amortises
                    "per_step_value": round(cells * e2e_steps / t_loop / 1e6, 1),
                    "per_step_d2h_bytes": d2h_step,
                    "create_read_destroy_s": round(e2e_s - t_loop, 4),
                    "api": "fpd_create, fpd_export_beads(4), per step fpd_step(1) + fpd_take_beads of the previous "
                           "step (the bead phase writes each table into a host ring), fpd_read_fields into page-locked "
                           "host buffers allocated before the timed region, fpd_destroy"},
            "clocks": clocks,
            "mass_after": diag[0],
            "accuracy": accuracy,
            "batched": batched,
            "fp16": fp16,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(
                cfg, budget_s=args.cpu_seconds,
                gpu_run=lambda n: gpu_state(fpd, cfg, args.precision, variant, n, stream))
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ CPU oracle
def cpu_baseline(cfg: dict, budget_s: float = 12.0, steps: int | None = None, gpu_run=None) -> dict:
    """The FP64 oracle, as it stands, on this host's cores: whole time steps of
    the same workload until about budget_s seconds (or a fixed step count).
    gpu_run(n), if given, returns the GPU's (u_x, u_y, R) after n steps of the
    timed configuration; they are compared with the oracle's state after its
    timed steps."""
    import oracle
    cores = os.cpu_count() or 1
    o = oracle.Sim(dict(cfg, threads=cores))
    cells = cfg["nx"] * cfg["ny"]
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and (el >= budget_s or n >= 1000)):
            break
    out = {"value": round(cells * n / el / 1e6, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": f"{n} full steps of {cfg['name']} ({cells} cells) in {el:.1f} s"}
    if gpu_run is not None:
        ux, uy, R = gpu_run(n)
        oux, ouy, _ = o.fields()
        oR = o.beads()[0]
        ou = np.concatenate([oux.ravel(), ouy.ravel()])
        out["gpu_vs_oracle"] = {
            "steps": n, "what": "the timed configuration (precision, sweep variant, graph chunks) on the GPU",
            "u_rel_l2": float(np.linalg.norm(np.concatenate([ux.ravel(), uy.ravel()]) - ou) / np.linalg.norm(ou)),
            "R_rel_l2": float(np.linalg.norm(R - oR) / np.linalg.norm(oR)),
            "bead_max_dR": float(np.abs(R - oR).max())}
    # the same oracle on one thread (the canonical single-core baseline), a
    # shorter sample
    o1 = oracle.Sim(dict(cfg, threads=1))
    t0 = time.perf_counter()
    n1 = 0
    while n1 < 1000 and time.perf_counter() - t0 < budget_s / 2:
        o1.step(1)
        n1 += 1
    el1 = time.perf_counter() - t0
    out["single_thread"] = {"value": round(cells * n1 / el1 / 1e6, 3), "unit": "MLUPS", "cores": 1,
                            "sample": f"{n1} full steps in {el1:.1f} s"}
    return out


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    from paper_2212_14153_gb300 import workloads
    import oracle
    oracle.build()
    cfg = workloads.two_fiber_large(precision=args.precision)
    cores = os.cpu_count() or 1
    o = oracle.Sim(dict(cfg, threads=cores))
    cells = cfg["nx"] * cfg["ny"]
    # each reference step is one full oracle time step of the same workload
    ref_steps = max(1, min(args.steps, args.ref_steps))
    ref_warm = max(0, min(args.warmup, 3))
    o.step(ref_warm)
    t0 = time.perf_counter()
    o.step(ref_steps)
    el = time.perf_counter() - t0
    v = cells * ref_steps / el / 1e6
    line = {
        "metric": "MLUPS (million lattice-cell updates per second) of the FPD-MRT step",
        "value": round(v, 3), "unit": "MLUPS", "n_gpus": world, "steps": ref_steps, "warmup": ref_warm,
        "ms_per_step": el * 1e3 / ref_steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": cfg["name"], "nx": cfg["nx"], "ny": cfg["ny"], "fibers": cfg["n_fibers"],
                   "beads_per_fiber": cfg["n_beads"], "storage": "f64 (A/B arrays)"},
        "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{ref_steps} full steps of {cfg['name']} after {ref_warm} warm-up"},
        "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ sweep / serving
def run_sweep(args, rank: int, world: int):
    """Batched sweep: independent instances (H ~ U{32..256}, width 2H, C, Re,
    K, a, N drawn as in the shape-diagram sweep) advanced by one batched
    launch pair per step, against the plain loop that runs the same instances
    one at a time with the same kernels and precision."""
    import torch
    from paper_2212_14153_gb300 import build, fpd, serve, workloads
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    inst = workloads.batched_sweep(n=args.instances, seed=4 + rank, precision=args.precision)
    cells = [c["nx"] * c["ny"] for c in inst]
    stream = torch.cuda.Stream()
    S, W = args.steps, args.warmup
    pool = sum(serve.state_bytes(c, args.precision) + 4096 for c in inst)
    nbeads = sum(c["n_beads"] * c["n_fibers"] for c in inst)
    b = fpd.Batch(args.precision, len(inst), pool, nbeads, stream=stream.cuda_stream)
    T = 64  # steps per variant for the launch-shape autotuning below
    nvar = fpd.fpd_sweep_variants()
    for c in inst:
        b.add(c, nvar * (T + 8) + W + S)
    variant_ms = []
    for v in range(nvar):
        b.set_tuning(v)
        b.run(8)
        b.sync()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        b.run(T)
        a1.record(stream)
        a1.synchronize()
        variant_ms.append(a0.elapsed_time(a1) / T)
    variant = int(min(range(nvar), key=lambda i: variant_ms[i])) if args.variant == "auto" else int(args.variant)
    b.set_tuning(variant)
    b.run(W)
    b.sync()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    done = 0
    while done < S:
        d = b.run(S - done)
        if d == 0:
            break
        done += d
    ev1.record(stream)
    ev1.synchronize()
    t_batch = ev0.elapsed_time(ev1) * 1e-3
    b.close()
    batched = sum(cells) * S / t_batch / 1e6
    # plain loop: each instance alone, one after the other
    t_plain = 0.0
    for c in inst:
        sim = fpd.Simulation(c, stream=stream.cuda_stream)
        sim.set_tuning(variant)
        sim.step(W)
        sim.sync()
        ev0.record(stream)
        sim.step(S)
        ev1.record(stream)
        ev1.synchronize()
        t_plain += ev0.elapsed_time(ev1) * 1e-3
        sim.close()
    plain = sum(cells) * S / t_plain / 1e6
    line = {
        "metric": "aggregate MLUPS, batched sweep vs plain one-instance-at-a-time loop",
        "value": round(batched, 1), "unit": "MLUPS", "plain_loop": round(plain, 1),
        "speedup": round(batched / plain, 2), "n_gpus": 1, "steps": S, "warmup": W,
        "higher_is_better": True, "dtype": {0: "f64", 1: "f32", 2: "f32"}[args.precision], "data": "synthetic",
        "config": {"workload": "batched_sweep", "instances": len(inst), "cells": sum(cells), "beads": nbeads,
                   "H": [min(c["ny"] for c in inst), max(c["ny"] for c in inst)],
                   "accuracy": "each instance bit-identical to its alone run",
                   "sweep_variant": variant, "variant_ms_per_step": [round(m, 4) for m in variant_ms]},
        "batched_s": t_batch, "plain_s": t_plain,
    }
    print(json.dumps(line), flush=True)
    return batched


def measure_capacity(reqs, precision, steps: int = 256, warm: int = 8) -> float:
    """Aggregate MLUPS of the batched engine with all of reqs resident."""
    import torch
    from paper_2212_14153_gb300 import fpd, serve
    stream = torch.cuda.Stream()
    pool = sum(serve.state_bytes(r, precision) + 4096 for r in reqs)
    nbeads = sum(r["n_beads"] * r["n_fibers"] for r in reqs)
    b = fpd.Batch(precision, len(reqs), pool, nbeads, stream=stream.cuda_stream)
    for r in reqs:
        b.add(r, warm + steps)
    b.run(warm)
    b.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.run(steps)
    e1.record(stream)
    e1.synchronize()
    b.close()
    return sum(r["nx"] * r["ny"] for r in reqs) * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6


def run_serve(args, rank: int, world: int):
    """Serving: Poisson arrivals of sweep-point requests at 0.5x and 1.2x the
    measured batched capacity; continuous batching under an HBM cap."""
    import torch
    from paper_2212_14153_gb300 import build, serve, workloads
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    out = []
    probe = workloads.serving_requests(args.serve_requests, 1.0, seed=5, steps_lo=args.serve_steps_lo,
                                       steps_hi=args.serve_steps_hi, precision=args.precision)
    work = np.mean([r["nx"] * r["ny"] * r["steps"] for r in probe])
    cap_mlups = args.capacity_mlups
    cap_how = "given (--capacity-mlups)"
    if cap_mlups <= 0:
        cap_mlups = measure_capacity(probe[:args.max_slots], args.precision)
        cap_how = f"measured: batched rate of the first {min(len(probe), args.max_slots)} requests resident at once"
    capacity = cap_mlups * 1e6 / work  # requests / s the batch can sustain
    for load in (0.5, 1.2):
        reqs = workloads.serving_requests(args.serve_requests, load * capacity, seed=5, steps_lo=args.serve_steps_lo,
                                          steps_hi=args.serve_steps_hi, precision=args.precision)
        pool = sum(serve.state_bytes(r, args.precision) + 4096 for r in reqs)
        nbeads = sum(r["n_beads"] * r["n_fibers"] for r in reqs)
        srv = serve.Server(args.precision, max_slots=args.max_slots, cap_bytes=args.cap_bytes,
                           pool_bytes=min(pool, args.cap_bytes), max_beads=nbeads, chunk=args.chunk)
        rs = [serve.Request(i, r, r["steps"], r["arrival_s"]) for i, r in enumerate(reqs)]
        res = srv.serve(rs)
        srv.close()
        res["load"] = load
        res["rate_per_s"] = load * capacity
        out.append(res)
    line = {
        "metric": "serving: p50/p99 time-to-result and aggregate MLUPS under Poisson arrivals",
        "value": round(out[0]["aggregate_mlups"], 1), "unit": "MLUPS", "n_gpus": 1,
        "higher_is_better": True, "dtype": {0: "f64", 1: "f32", 2: "f32"}[args.precision], "data": "synthetic",
        "config": {"workload": "serving", "requests": args.serve_requests,
                   "steps_per_request": [args.serve_steps_lo, args.serve_steps_hi], "chunk": args.chunk,
                   "cap_bytes": args.cap_bytes, "capacity_mlups": round(cap_mlups, 1), "capacity": cap_how,
                   "latency": "arrival to result on the host; admission happens at chunk boundaries, so it "
                              "includes up to one chunk of waiting"},
        "loads": out,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1, 2])
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10000)
    ap.add_argument("--accuracy-steps", type=int, default=200)
    ap.add_argument("--ref-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="two_fiber", choices=["two_fiber", "sweep", "serve"])
    ap.add_argument("--instances", type=int, default=512)
    ap.add_argument("--serve-steps-lo", type=int, default=50000)
    ap.add_argument("--serve-steps-hi", type=int, default=500000)
    ap.add_argument("--serve-requests", type=int, default=128)
    ap.add_argument("--cap-bytes", type=int, default=150 << 30)
    ap.add_argument("--max-slots", type=int, default=512)
    ap.add_argument("--chunk", type=int, default=500)
    ap.add_argument("--variant", default="auto",
                    help="sweep launch shape: auto (timed by the autotuner) or a variant number "
                         "below fpd_sweep_variants()")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and FP16 sub-measurements")
    ap.add_argument("--batched-instances", type=int, default=128)
    ap.add_argument("--batched-steps", type=int, default=64)
    ap.add_argument("--capacity-mlups", type=float, default=0.0,
                    help="serving capacity; 0 = measure the batched rate of the same requests first")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "sweep":
        run_sweep(args, rank, world)
    elif args.workload == "serve":
        run_serve(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
