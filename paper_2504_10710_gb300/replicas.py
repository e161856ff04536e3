"""Replica bookkeeping for multi-GPU runs.  Independent problems shard across
ranks with no data-path communication; ranks only meet at a barrier before
and after the timed region and agree on the slowest rank's time."""
from __future__ import annotations

import os


def rank_world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world: int) -> float:
    """The largest of every rank's value (the timed region ends when the
    slowest replica ends)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: float, seconds_per_rank: float, world: int) -> float:
    """Whole-job throughput: the units all ranks processed divided by the
    max-over-ranks time (weak scaling: every rank does the same work)."""
    return world * units_per_rank / max_over_ranks(seconds_per_rank, world)


def shard(items, rank: int, world: int):
    """Round-robin assignment of independent problems to ranks."""
    return [x for i, x in enumerate(items) if i % world == rank]
