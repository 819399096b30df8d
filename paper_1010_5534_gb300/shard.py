"""Sharding renders over ranks (one process per GPU).

Batched renders: views are independent problems (each view's quadtree is
refined on its own image), so a batch shards by view with no exchange on the
data path (weak scaling). Ranks take views round-robin (view v goes to rank v
mod world), which spreads views of similar cost evenly; after rendering, only
per-view summaries (counts and band fluxes, a few numbers per view) are
gathered.

One image: the paper (Section 2, parallelisation) distributes the pixels of
each ray-tracing sweep over the processors and gathers the traced values for
the refinement check. air_render_adaptive_sharded splits every sweep's new
rays into contiguous slices, one per rank, and calls back for the exchange;
`ray_slices` and `exchange_slices` are that exchange over torch.distributed
(an all-gather of one packed buffer per sweep).
"""
from __future__ import annotations


def shard_views(n_views: int, rank: int, world: int) -> list:
    """Indices of the views rank `rank` of `world` renders."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(range(rank, n_views, world))


def gather_summaries(local: dict, n_views: int, group=None) -> list:
    """All-gather per-view summaries {view index: summary} of every rank into a
    list ordered by view index (every rank receives the full list)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    out = [None] * n_views
    for p in parts:
        for k, v in p.items():
            if out[k] is not None:
                raise RuntimeError(f"view {k} rendered by two ranks")
            out[k] = v
    missing = [k for k, v in enumerate(out) if v is None]
    if missing:
        raise RuntimeError(f"views {missing} rendered by no rank")
    return out


def summary(result: dict) -> dict:
    """The small, host-side part of a render result that ranks exchange."""
    bf = result.get("band_flux")
    if bf is not None and hasattr(bf, "cpu"):
        bf = bf.cpu().tolist()
    return {k: result[k] for k in ("n_rays", "n_leaves", "n_steps", "n_sweeps") if k in result} | \
        ({"band_flux": list(bf)} if bf is not None else {})


def ray_slices(count: int, world: int) -> list:
    """Bounds [lo_r, hi_r) of the contiguous slice rank r traces out of
    `count` rays: lo_r = count r / world (integer division), as the library
    splits them."""
    if world < 1:
        raise ValueError("world must be >= 1")
    return [(count * r // world, count * (r + 1) // world) for r in range(world)]


def exchange_slices(arrays, rank: int, world: int, group=None) -> None:
    """All-gather the ray slices of one sweep in place. `arrays`: 1-D tensors
    of 4-byte elements (float32 or int32), all `count` long and on one device,
    of which this rank filled its slice (ray_slices); on return every rank's
    arrays hold every slice. The arrays are packed into one buffer per rank
    (padded to the longest slice) and exchanged with one all_gather; on a
    CUDA device with the NCCL backend the exchange stays on the device,
    otherwise it goes through host memory (gloo)."""
    import torch
    import torch.distributed as dist
    count = int(arrays[0].numel())
    sl = ray_slices(count, world)
    lo, hi = sl[rank]
    chunk = max(h - l for l, h in sl)
    if chunk == 0:
        return
    dev = arrays[0].device
    on_dev = dev.type == "cuda" and dist.get_backend(group) == "nccl"
    work = dev if on_dev else torch.device("cpu")
    na = len(arrays)
    mine = torch.zeros((na, chunk), dtype=torch.int32, device=work)
    for a, x in enumerate(arrays):
        mine[a, :hi - lo] = x[lo:hi].view(torch.int32).to(work)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    for r, (l, h) in enumerate(sl):
        if r == rank or h == l:
            continue
        for a, x in enumerate(arrays):
            x.view(torch.int32)[l:h] = parts[r][a, :h - l].to(dev)
