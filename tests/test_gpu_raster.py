"""Finest-level raster (air_render_raster, Section 2 step vi) against the
raster oracle on the GPU's own tree: nearest bit-exact, bilinear within FP32
rounding of the four products and three sums (2e-7 relative, plus 1e-7 of the
image maximum), for the three quantities, on mixed-level images."""
import numpy as np
import pytest

import paper_1010_5534_gb300 as air
import scenes
from oracle import raster as R

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def grid():
    air.build()
    s = scenes.cone_shock_amr(1, n_base=32, brick=8, levels=2, n_bands=3, e_lo=0.5, kappa0=0.4,
                              thickness=0.08)
    g = air.Grid(s)
    yield s, g
    g.close()


def np_(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("vidx", [0, 1])
def test_raster_matches_oracle(grid, vidx):
    sc, g = grid
    v = scenes.axis_view("+z") if vidx == 0 else scenes.random_views(6, 1)[0]
    n0, Lm = 12, 3
    r = g.render_adaptive(v, n0, Lm, 0.3, include_interior=True)
    lv, i, j = np_(r["level"]), np_(r["i"]), np_(r["j"])
    assert len(np.unique(lv)) > 2          # mixed levels
    vals = {"p": np_(r["p"]), "N": np_(r["coldens"]), "I": np_(r["intensity"])[2]}
    for q, val in vals.items():
        for mode in ("nearest", "bilinear"):
            out = np_(g.raster(q, band=2, mode=mode))
            want = R.raster(lv, i, j, val.astype(np.float64), n0, Lm, mode)
            assert out.shape == want.shape == (n0 << Lm, n0 << Lm)
            if mode == "nearest":
                assert (out == want.astype(np.float32)).all(), q
            else:
                tol = 2e-7 * np.abs(want) + 1e-7 * np.abs(want).max()
                bad = np.abs(out - want) > tol
                assert not bad.any(), (q, int(bad.sum()))
    # a host destination gives the same bits
    host = g.raster("p", mode="bilinear", mem="host")
    assert (host.numpy() == np_(g.raster("p", mode="bilinear"))).all()


def test_raster_errors(grid):
    sc, g = grid
    v = scenes.axis_view("+x")
    g.render_adaptive(v, 8, 2, 0.3)
    out = torch.empty(10, dtype=torch.float32, device="cuda")
    L = air.lib()
    import ctypes as C
    assert L.air_render_raster(g._h, 1, 0, 1, C.c_void_p(out.data_ptr()), 10) == air.AIR_ERR_CAPACITY
    assert L.air_render_raster(g._h, 0, 7, 1, C.c_void_p(out.data_ptr()), 1 << 20) == air.AIR_ERR_ARG
    assert L.air_render_raster(g._h, 5, 0, 1, C.c_void_p(out.data_ptr()), 1 << 20) == air.AIR_ERR_ARG
    assert L.air_render_raster(g._h, 1, 0, 9, C.c_void_p(out.data_ptr()), 1 << 20) == air.AIR_ERR_ARG
    # a batched render replaces the single-view tree
    g.render_batch([v, scenes.axis_view("+y")], 8, 2, 0.3)
    assert L.air_render_raster(g._h, 1, 0, 1, C.c_void_p(out.data_ptr()), 1 << 20) == air.AIR_ERR_ARG
