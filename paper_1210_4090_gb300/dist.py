"""Multi-rank helpers for one node: sharding independent instances, the final
gather of the sweep's per-instance H-bar estimates, and the timing reduction
of a benchmark step (max time, summed work over ranks).

The scheme's single grid does not shard in this library (each rank runs a
replica); the batched sweep shards by instance (instances are independent
grids; Sec. 4.1 distributivity makes every convolution block independent),
with no collective on the data path -- only the gather of the H-bar values
at the end and the timing reduction below.
"""
from __future__ import annotations

import heapq


def lpt_assign(weights, world: int):
    """Longest-processing-time-first assignment of items to `world` ranks:
    items by decreasing weight (ties: lower index first), each to the rank
    with the least load so far (ties: lower rank).  Returns the owner rank of
    every item.  Graham's bound: the largest load is at most 4/3 - 1/(3 world)
    times the optimal largest load."""
    if world < 1:
        raise ValueError("bad world")
    order = sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i))
    heap = [(0.0, r) for r in range(world)]
    owner = [0] * len(weights)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + float(weights[i]), r))
    return owner


def shard(items, rank: int, world: int, weights=None):
    """This rank's items, in their original order.  With weights (the work of
    each item, e.g. N_i^2 points of an instance), by LPT over the ranks;
    without, every world-th item starting at rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    if weights is None:
        return items[rank::world]
    if len(weights) != len(items):
        raise ValueError("one weight per item")
    owner = lpt_assign(weights, world)
    return [it for it, o in zip(items, owner) if o == rank]


def shard_indices(n: int, rank: int, world: int, weights=None):
    """shard() of range(n): the indices of this rank's items."""
    return shard(list(range(n)), rank, world, weights)


def gather_rows(local_rows, local_index, n: int, device=None):
    """Every rank's rows of an (n, k) float64 table, each rank holding the rows
    local_rows[j] of items local_index[j], gathered on every rank in item
    order (all_gather of fixed-size buffers; identity without a process
    group).  Returns a numpy array (n, k)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    rows = np.asarray(local_rows, dtype=np.float64).reshape(len(local_index), -1)
    k = rows.shape[1] if rows.size else 0
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        out = np.zeros((n, k))
        out[np.asarray(local_index, dtype=np.int64)] = rows
        return out
    world = dist.get_world_size()
    kk = torch.tensor([k], dtype=torch.int64, device=device)
    dist.all_reduce(kk, op=dist.ReduceOp.MAX)
    k = int(kk.item())
    # every rank sends n rows (index + k values), NaN-padded where it owns none
    buf = np.full((n, k + 1), np.nan)
    for j, i in enumerate(local_index):
        buf[j, 0] = float(i)
        buf[j, 1:] = rows[j]
    t = torch.tensor(buf, dtype=torch.float64, device=device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    out = np.full((n, k), np.nan)
    for part in parts:
        p = part.cpu().numpy()
        for row in p:
            if not np.isnan(row[0]):
                out[int(row[0])] = row[1:]
    return out


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
