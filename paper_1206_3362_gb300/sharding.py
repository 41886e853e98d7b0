"""Frame sharding across ranks.

Frames are independent units of work, so N ranks (one GPU each) decode
disjoint frame sets with no collective on the data path; the only collective
is the max over ranks of the timed region, which makes the reported time that
of the slowest rank.
"""
from __future__ import annotations


def shard_range(n_frames: int, rank: int, world: int):
    """Contiguous [lo, hi) share of rank in world (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_frames, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def frame_seed(seed: int, rank: int) -> int:
    """Seed of a rank's own synthetic frames (weak scaling: every rank makes
    and decodes its own batch)."""
    return seed * 1009 + rank


def max_over_ranks(value: float, device=None) -> float:
    """Max of a scalar over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
