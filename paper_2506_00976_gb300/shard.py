"""Sharding of independent pairs across ranks (one process per GPU).

Pairs share nothing, so the method shards by pair with no collective on the
data path: each rank runs its own pairs, and ranks only agree on timing (a
barrier and a maximum).  For pairs of uneven size the assignment is the
longest-processing-time rule on the per-pair work, which is dominated by the
N^{2d} = N^4 pixel pairs of the c-transform and of C-bar.
"""
from __future__ import annotations

from typing import List, Sequence


def pair_cost(N: int) -> float:
    """Relative work of one pair on an N x N grid (pixel pairs, N^4)."""
    return float(N) ** 4


def lpt_shards(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Split pair indices across `world` ranks: largest pair first, each to the
    least loaded rank (ties to the lowest rank).  Every index appears once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda t: (-pair_cost(sizes[t]), t))
    loads = [0.0] * world
    shards: List[List[int]] = [[] for _ in range(world)]
    for t in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        shards[r].append(t)
        loads[r] += pair_cost(sizes[t])
    for s in shards:
        s.sort()
    return shards


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (identity
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
