"""Rank bookkeeping for multi-GPU runs of independent work (weak scaling).

The workloads shard without any data-path collective: every rank runs its own
copy of the work on its own GPU.  The only cross-rank operations are a barrier
before the timed region and a MAX reduction of the per-rank elapsed time, so
the job's throughput is (units on all ranks) / (slowest rank's time).
Works with any torch.distributed backend (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds_this_rank: float) -> tuple[float, float]:
    """(whole-job units per second, slowest rank's seconds) for weak scaling."""
    import torch.distributed as dist
    n = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    slowest = max_over_ranks(seconds_this_rank)
    return n * units_per_rank / slowest, slowest
