"""Host-side multi-GPU helpers: the path shards by view, so ranks split the views and never exchange
data; only the timing is reduced (max over ranks) and results may be gathered on rank 0."""
from __future__ import annotations


def shard_views(n_views: int, rank: int, world: int) -> list[int]:
    """Views owned by ``rank``: a contiguous block, sizes differing by at most one."""
    if not (0 <= rank < world) or n_views < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_views, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def max_over_ranks(value: float, device=None) -> float:
    """Largest ``value`` over all ranks of the default process group (the value itself without one)."""
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
