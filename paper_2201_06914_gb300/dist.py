"""Shot sharding across ranks (one process per GPU).  Shots are independent, so a survey
is split into contiguous shot ranges with no data-path collective; the only reductions are
the timing (max over ranks) and, when the stacked gradient of the whole survey is wanted,
one sum of an N-float image."""
from __future__ import annotations


def shot_range(nshots_total: int, rank: int, world: int) -> range:
    """Contiguous block of shots owned by `rank` (sizes differ by at most one)."""
    base, extra = divmod(nshots_total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_image(g):
    """Stacked gradient over ranks (in place): the one exchange of the shot-parallel path."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(g, op=dist.ReduceOp.SUM)
    return g
