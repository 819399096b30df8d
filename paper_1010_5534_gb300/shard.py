"""Sharding batched renders over ranks (one process per GPU).

Views are independent problems: each view's quadtree is refined on its own
image, so a batch shards by view with no exchange on the data path (weak
scaling). Ranks take views round-robin (view v goes to rank v mod world), which
spreads views of similar cost evenly; after rendering, only per-view summaries
(counts and band fluxes, a few numbers per view) are gathered.
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
