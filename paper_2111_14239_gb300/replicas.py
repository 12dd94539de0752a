"""Replica (weak-scaling) bookkeeping for multi-GPU runs.

The rounded-KLT path has no exchange step: every block, and so every image, is
independent.  Each rank therefore processes its own images with no collective on
the data path; the only collective is on the timing scalar, so that whole-job
throughput = units processed by all ranks / slowest rank's time.
"""
from __future__ import annotations

import os


def world() -> tuple:
    """(rank, world_size, local_rank) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def image_seeds(base_seed: int, n_per_rank: int, rank: int) -> list:
    """Seeds of this rank's images: rank r takes base + r*n .. base + r*n + n - 1, so
    ranks never share an image and rank 0 alone reproduces the single-GPU workload
    (the rule lives with the input generators, synth_inputs.rank_seeds)."""
    import synth_inputs
    return synth_inputs.rank_seeds(base_seed, n_per_rank, rank)


def shard(n_items: int, rank: int, world_size: int) -> range:
    """Contiguous near-equal split of n_items over ranks (strong-scaling helper)."""
    q, rem = divmod(n_items, world_size)
    lo = rank * q + min(rank, rem)
    return range(lo, lo + q + (1 if rank < rem else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Max of a scalar over the process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world_size: int, seconds_max: float) -> float:
    """Whole-job rate: all ranks' units over the slowest rank's time."""
    return units_per_rank * world_size / seconds_max
