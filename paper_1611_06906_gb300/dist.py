"""Multi-GPU helpers: one process per GPU, images sharded across ranks.

The filter has no exchange step between images, so a batch shards across
ranks with no collective on the data path (weak scaling: every rank filters its
own batch).  The only collectives are the timing barrier and the max-over-ranks
reduction of the measured time.
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_units: int, rank: int, world: int):
    """Contiguous, balanced range [lo, hi) of n_units owned by `rank`."""
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_seed(seed0: int, rank: int, stride: int = 1000) -> int:
    """Seed of rank `rank`'s batch (weak scaling: every rank has its own images)."""
    return seed0 + stride * rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
