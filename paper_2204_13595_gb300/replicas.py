"""Replica bookkeeping of multi-GPU runs.

The force step does not shard here (one GPU per system: "replicas only"):
under torchrun every rank steps its own independent system, seeded from the
base seed and its rank, with no collective on the data path.  The only
collectives are the timing ones: a barrier on both sides of the timed region
and the maximum of the per-rank times, from which the whole-job throughput is
formed (weak scaling: the work per rank is fixed).
"""
from __future__ import annotations

import os


def world():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's replica: distinct per rank, the base seed on rank 0."""
    return int(base_seed) + int(rank)


def barrier(world_size: int):
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world_size: int, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (the slowest rank's time)."""
    if world_size <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(world_size: int, units_per_rank: float, max_ms: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return world_size * float(units_per_rank) * 1e3 / float(max_ms)
