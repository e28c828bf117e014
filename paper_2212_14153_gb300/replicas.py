"""Replica placement for several GPUs (one process per GPU).

Instances of the method are independent (sweep points, requests), so the
multi-GPU form shares the list of instances out across ranks and never
exchanges data on the path: a rank runs its own instances; only the timing
(max over ranks) and the counts (sum over ranks) are combined, on the host
side of each measurement.
"""
from __future__ import annotations


def shard(items: list, rank: int, world: int) -> list:
    """Round-robin share of `items` for `rank` of `world` (every item once)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    return items[rank::world]


def _reduce(value: float, op: str) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(value: float) -> float:
    """Slowest rank's value (the job's time)."""
    return _reduce(value, "max")


def sum_over_ranks(value: float) -> float:
    """Total over ranks (work done by the whole job)."""
    return _reduce(value, "sum")


def job_rate(units_per_rank: float, seconds_per_rank: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return sum_over_ranks(units_per_rank) / max_over_ranks(seconds_per_rank)
