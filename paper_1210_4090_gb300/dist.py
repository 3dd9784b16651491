"""Multi-rank helpers for one node: sharding independent instances and the
timing reduction of a benchmark step (max time, summed work over ranks).

The scheme's single grid does not shard in this library (each rank runs a
replica); the batched sweep shards by instance (instances are independent,
Sec. 4.1 distributivity), with no collective on the data path -- only the
timing reduction below.
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Every world-th item starting at rank (round-robin keeps the size mix)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return items[rank::world]


def reduce_step(total_ms: float, updates: float, device=None):
    """(max total_ms, sum updates) over the ranks of the default process group
    (identity when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(updates)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
