"""Host logic of a multi-GPU run: one replica per rank, no data-path exchange.

The right-hand sides of one operator (and the independent instances of the
batched workload) need no communication while they are solved, so N GPUs run
N replicas of the benchmark's problem, each with its own seeded instance
(weak scaling).  The only collectives are outside the solve: a barrier
around the timed region and a MAX of the timings, so that the reported time
is the slowest rank's.  These helpers take the process group and the device
of the reduction tensor as arguments, so the same code runs with NCCL on GPUs
and with gloo on CPU (tests).
"""
from __future__ import annotations

import os


def rank_env():
    """(world size, global rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_instance(rank: int) -> int:
    """Seed instance of the workload solved by `rank` (distinct per rank)."""
    return rank


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest value of x over all ranks (x itself without a group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The sum of x over all ranks (x itself without a group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_rate(units_per_rank: float, seconds_max: float, dist=None, device="cpu") -> float:
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time."""
    return sum_over_ranks(units_per_rank, dist, device) / seconds_max
