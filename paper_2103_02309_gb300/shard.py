"""Host-side work split for N replicas (one process per GPU).

Rays are independent (one walk per ray, Sec. 7) and every replica holds
the whole mesh, so the multi-GPU logic is on the host: which meshes of a
batch each rank traces, which pixel tiles of one frame each rank traces,
the gather of a frame's hits to rank 0, and the max-over-ranks step time.
The walk itself has no exchange step.
"""
from __future__ import annotations

GAMMA = 0x9E3779B97F4A7C15   # SplitMix64's increment (Steele, Lea & Flood, OOPSLA 2014)
TILE_RAYS = 32               # camera rays are stored in 8x4-pixel warp tiles


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


def tile_range(n_rays: int, world: int, rank: int, tile: int = TILE_RAYS) -> tuple[int, int]:
    """The contiguous rays [lo, hi) of one frame that `rank` traces: whole
    warp tiles (`tile` rays each, the last one possibly ragged), split as
    evenly as whole tiles allow and in rank order, so that the ranks' ranges
    cover the frame once and concatenate in pixel-tile order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    tiles = (n_rays + tile - 1) // tile
    lo_t = tiles * rank // world
    hi_t = tiles * (rank + 1) // world
    return min(n_rays, lo_t * tile), min(n_rays, hi_t * tile)


def shard_seed(seed: int, first_ray: int, per_hit: int) -> int:
    """The seed that makes a rank's secondary rays equal the whole frame's.

    The generators draw number c of stream `seed` as mix64(seed + (c+1) *
    GAMMA) (SplitMix64 used as a counter-based generator), with counter
    c = 2 (i * per_hit + k) + j for hit i of the buffer.  A rank whose buffer
    starts at frame ray `first_ray` counts from i = 0, so it shifts the seed
    by 2 * first_ray * per_hit increments instead of the counter."""
    return (int(seed) + 2 * int(first_ray) * int(per_hit) * GAMMA) % (1 << 64)


def gather_rows(local, world: int, rank: int, device=None):
    """Rank 0 gets every rank's rows (a [m_r, ...] tensor each, m_r may
    differ) concatenated in rank order; the other ranks get None.  Without a
    process group the rows are returned as they are."""
    import torch
    import torch.distributed as dist
    if world == 1 or not (dist.is_available() and dist.is_initialized()):
        return local
    m = torch.tensor([local.shape[0]], dtype=torch.int64, device=device)
    counts = [torch.zeros_like(m) for _ in range(world)]
    dist.all_gather(counts, m)
    counts = [int(c.item()) for c in counts]
    width = max(counts)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    if rank != 0:
        return None
    return torch.cat([p[:c] for p, c in zip(parts, counts)])
