"""Batched rendering sharded over ranks (world size 2, gloo, CPU): every view
is rendered by exactly one rank, the gathered summaries equal a single-process
render of all views, and a rank that raises is reported, not hung. Ranks
render with the FP64 oracle here (no GPU); the CUDA path uses the same
sharding and gather."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1010_5534_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _views():
    import scenes
    return scenes.random_views(12, 5)


def _render(o, v):
    t = o.air(v, 8, 2, 0.4)
    return {"n_rays": int(t["n_nodes"]), "n_leaves": int(t["n_leaves"]), "n_steps": int(t["n_steps"]),
            "n_sweeps": int(t["n_sweeps"]), "band_flux": [float(x) for x in t["band_flux"]]}


def _worker(rank, world, port, q, fail_rank):
    import torch.distributed as dist
    import oracle
    import scenes
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = scenes.cone_shock_amr(2, n_base=16, brick=4, levels=1, n_bands=2, e_lo=0.5)
        o = oracle.Oracle(sc)
        vs = _views()
        mine = shard.shard_views(len(vs), rank, world)
        if rank == fail_rank:
            raise RuntimeError("injected failure")
        local = {k: _render(o, vs[k]) for k in mine}
        allv = shard.gather_summaries(local, len(vs))
        q.put((rank, mine, allv))
    except Exception as e:  # report on the host; never leave a peer waiting on us
        q.put((rank, "error", str(e)))
    finally:
        dist.destroy_process_group()


def _run(world, fail_rank=-1, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in ps:
        p.start()
    out = []
    for _ in range(world):
        out.append(q.get(timeout=timeout))
    for p in ps:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return sorted(out, key=lambda x: x[0])


def test_shard_views_partition():
    for n in (0, 1, 5, 64):
        for w in (1, 2, 3, 8):
            got = sorted(sum((shard.shard_views(n, r, w) for r in range(w)), []))
            assert got == list(range(n))
    with pytest.raises(ValueError):
        shard.shard_views(4, 2, 2)


def test_two_ranks_match_one_process():
    import oracle
    import scenes
    out = _run(2)
    sc = scenes.cone_shock_amr(2, n_base=16, brick=4, levels=1, n_bands=2, e_lo=0.5)
    o = oracle.Oracle(sc)
    ref = [_render(o, v) for v in _views()]
    (r0, m0, a0), (r1, m1, a1) = out
    assert sorted(m0 + m1) == list(range(5)) and not set(m0) & set(m1)
    assert a0 == a1
    for got, exp in zip(a0, ref):
        assert got["n_rays"] == exp["n_rays"] and got["n_steps"] == exp["n_steps"]
        np.testing.assert_array_equal(got["band_flux"], exp["band_flux"])


def test_failing_rank_is_reported():
    out = _run(2, fail_rank=1, timeout=120)
    assert out[1][1] == "error" and "injected" in out[1][2]
    # the healthy rank either finished its gather or reports the broken group
    assert out[0][1] == "error" or isinstance(out[0][1], list)


# ---- one image, rays of every sweep split over ranks --------------------------
def _slice_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = []
        for count in (0, 1, 2, 5, 17, 1000):
            full_f = torch.arange(count, dtype=torch.float32) * 1.5 + 0.25
            full_i = torch.arange(count, dtype=torch.int32) * 7 - 3
            f = torch.full((count,), float("nan"))
            i = torch.full((count,), -99, dtype=torch.int32)
            lo, hi = shard.ray_slices(count, world)[rank]
            f[lo:hi] = full_f[lo:hi]
            i[lo:hi] = full_i[lo:hi]
            shard.exchange_slices([f, i], rank, world)
            out.append(bool(torch.equal(f, full_f)) and bool(torch.equal(i, full_i)))
        q.put((rank, out))
    except Exception as e:
        q.put((rank, "error: " + str(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ray_slice_exchange(world):
    """exchange_slices (the host side of air_render_adaptive_sharded) fills
    every rank's arrays with every slice, for counts below, at and above the
    number of ranks."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_slice_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
    for rank, out in res:
        assert out == [True] * 6, (rank, out)


def test_ray_slices_cover_each_ray_once():
    for count in (0, 1, 3, 10, 1001):
        for world in (1, 2, 3, 8):
            sl = shard.ray_slices(count, world)
            assert sl[0][0] == 0 and sl[-1][1] == count
            assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
            assert max(h - l for l, h in sl) - min(h - l for l, h in sl) <= 1
