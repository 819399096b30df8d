"""One image over two processes (air_render_adaptive_sharded): each rank
traces its slice of every sweep's rays and the slices are exchanged over gloo
(the paper's Section 2 parallelisation: trace distributed, gather for the
refinement check). Both ranks share the one GPU; their kernels never wait on
each other (the exchange goes through the host). Every rank's image must be
bitwise equal to the single-process render."""
import os
import socket
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import paper_1010_5534_gb300 as air
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
KEYS = ("level", "i", "j", "is_leaf", "coldens", "intensity", "p", "band_flux")
CASES = [  # (scene kwargs, view, n0, Lm, xi_crit)
    (dict(seed=3, n_base=32, brick=8, levels=2, n_bands=3, e_lo=0.5), "+z", 16, 3, 0.3),
    (dict(seed=5, n_base=32, brick=8, levels=2, n_bands=2, e_lo=0.5), "oblique", 13, 3, 0.4),
]


def _scene_view(case):
    kw, vname, n0, Lm, xc = CASES[case]
    sc = scenes.cone_shock_amr(**kw)
    v = scenes.axis_view("+z") if vname == "+z" else scenes.random_views(4, 1)[0]
    return sc, v, n0, Lm, xc


def _child(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        res = {}
        for case in range(len(CASES)):
            sc, v, n0, Lm, xc = _scene_view(case)
            g = air.Grid(sc)
            r = g.render_adaptive_sharded(v, n0, Lm, xc, include_interior=True)
            for k in KEYS:
                res[f"{case}_{k}"] = r[k].cpu().numpy()
            res[f"{case}_n"] = np.array([r["n_rays"], r["n_steps"], r["n_sweeps"]])
            g.close()
        np.savez(out_path, **res)
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_sharded_image_equals_single_process():
    air.build()
    world = 2
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        outs = [os.path.join(d, f"rank{r}.npz") for r in range(world)]
        code = ("import sys; sys.path.insert(0, {root!r}); sys.path.insert(0, {here!r}); "
                "import test_gpu_shard_image as t; t._child({rank}, {world}, {port}, {out!r})")
        procs = [subprocess.Popen([sys.executable, "-c",
                                   code.format(root=os.path.dirname(HERE), here=HERE, rank=r,
                                               world=world, port=port, out=outs[r])])
                 for r in range(world)]
        try:
            for p in procs:
                assert p.wait(timeout=600) == 0
        finally:
            for p in procs:
                if p.poll() is None:
                    p.kill()
        got = [dict(np.load(o)) for o in outs]
    for case in range(len(CASES)):
        sc, v, n0, Lm, xc = _scene_view(case)
        g = air.Grid(sc)
        ref = g.render_adaptive(v, n0, Lm, xc, include_interior=True)
        for rank in range(world):
            for k in KEYS:
                x = got[rank][f"{case}_{k}"]
                y = ref[k].cpu().numpy()
                assert x.shape == y.shape and (x == y).all(), (case, rank, k)
            assert list(got[rank][f"{case}_n"]) == [ref["n_rays"], ref["n_steps"], ref["n_sweeps"]]
        g.close()


def test_sharded_bad_arguments():
    air.build()
    import ctypes as C
    sc = scenes.wind_shell_uniform(0, n=16)
    g = air.Grid(sc)
    v = scenes.axis_view("+z")
    p = air.Params(8, 2, 0.5, 0, 0, -1, 0)
    im = air.Image()
    im.mem = air.AIR_DEVICE
    im.capacity = 0
    for rank, world, fn in ((2, 2, None), (-1, 2, None), (0, 0, None), (0, 2, None)):
        sh = air.Shard(rank, world, fn if fn else air.EXCHANGE_FN(), None)
        st = air.lib().air_render_adaptive_sharded(g._h, C.byref(air._view(v)), C.byref(p),
                                                   C.byref(sh), C.byref(im))
        assert st == air.AIR_ERR_ARG, (rank, world)
    # world 1: no exchange needed, same image as the plain render
    sh = air.Shard(0, 1, air.EXCHANGE_FN(), None)
    r = g.render_adaptive(v, 8, 2, 0.5)
    buf = g.alloc_image(r["n_out"], "device", ("coldens",))
    im = g._image_of(buf, "device")
    assert air.lib().air_render_adaptive_sharded(g._h, C.byref(air._view(v)), C.byref(p),
                                                 C.byref(sh), C.byref(im)) == air.AIR_OK
    assert (buf["coldens"][:r["n_out"]] == r["coldens"]).all()
    g.close()
