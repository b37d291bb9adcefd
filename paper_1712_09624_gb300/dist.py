"""Multi-GPU host logic: independent tables per rank, no data-path collective.

Each rank serves its own table (the paper's one private table per core,
Sec. 2 and Sec. 5.3, one GPU per rank here); the only collective is the
timing reduction of the benchmark: the job's time is the slowest rank's, and
its throughput counts the work of all ranks.
"""

from __future__ import annotations

import os

import torch


def rank_info() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's table and traffic: ranks draw disjoint workloads."""
    return seed + 1000 * rank


def max_over_ranks(seconds: float, device=None) -> float:
    """The slowest rank's time (all_reduce MAX); the value itself when not distributed."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, steps: int, seconds: float, world: int) -> float:
    """Units of all ranks per second over the slowest rank's time."""
    return world * units_per_rank * steps / seconds
