"""Host-side work split for N independent replicas (one process per GPU).

Rays are independent and every replica holds the whole mesh, so the only
multi-GPU logic is on the host: which meshes of a batch each rank traces,
and the max-over-ranks step time.  There is no exchange step and no
collective on the data path; the one collective here reduces a timing.
"""
from __future__ import annotations


def lpt_assign(costs, world: int) -> list[int]:
    """Rank of every item under longest-processing-time-first scheduling.

    Items are taken in order of decreasing cost (ties by index) and each goes
    to the rank with the smallest load so far (ties by rank).  The largest
    load is at most 4/3 of the optimum (Graham, "Bounds on multiprocessing
    timing anomalies", 1969).
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    rank = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        rank[i] = r
        load[r] += float(costs[i])
    return rank


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over the ranks of the default process group
    (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
