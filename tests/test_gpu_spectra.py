"""Streamed spectra (air_render_adaptive_spectra): every node's spectrum goes
to page-locked host memory sweep by sweep, the device quadtree keeping only
the band-summed intensity and column density. Same kernels and rays as the
resident path, so every output is bitwise equal to air_render_adaptive's."""
import ctypes as C

import numpy as np
import pytest

import paper_1010_5534_gb300 as air
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def grid():
    air.build()
    s = scenes.cone_shock_amr(1, n_base=32, brick=8, levels=2, n_bands=6, e_lo=0.5, kappa0=0.4,
                              thickness=0.08)
    g = air.Grid(s)
    yield s, g
    g.close()


def np_(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("vidx", [0, 1])
def test_streamed_spectra_equal_resident(grid, vidx):
    sc, g = grid
    v = scenes.axis_view("-y") if vidx == 0 else scenes.random_views(12, 1)[0]
    ref = g.render_adaptive(v, 16, 3, 0.3, include_interior=True)
    got, spec = g.render_adaptive_spectra(v, 16, 3, 0.3)
    assert spec.is_pinned() and spec.shape == (sc.n_bands, ref["n_out"])
    assert got["n_out"] == ref["n_out"] and got["n_sweeps"] == ref["n_sweeps"] > 1
    for k in ("level", "i", "j", "is_leaf", "coldens", "p", "band_flux"):
        assert (np_(got[k]) == np_(ref[k])).all(), k
    assert (spec.numpy() == np_(ref["intensity"])).all()
    assert got["n_steps"] == ref["n_steps"]
    # the tree has no intensities now: raster of p works, of a band does not
    g.raster("p")
    with pytest.raises(air.AirError):
        g.raster("I", band=1)
    # a resident render afterwards gets its intensities back
    again = g.render_adaptive(v, 16, 3, 0.3, include_interior=True)
    assert (np_(again["intensity"]) == np_(ref["intensity"])).all()


def test_streamed_spectra_capacity_and_arguments(grid):
    sc, g = grid
    v = scenes.axis_view("+z")
    ref = g.render_adaptive(v, 16, 3, 0.3, include_interior=True)
    # too small a host array: capacity error with the node count, then a retry fits
    got, spec = g.render_adaptive_spectra(v, 16, 3, 0.3, spectra_cap=300)
    assert spec.shape[1] == ref["n_out"] > 300
    assert (spec.numpy() == np_(ref["intensity"])).all()
    L = air.lib()
    p = air.Params(16, 3, 0.3, 0, 0, -1, 1)
    im, out = g._alloc(ref["n_out"], "device", ("level", "band_flux"))
    pageable = np.zeros((sc.n_bands, ref["n_out"]), np.float32)
    assert L.air_render_adaptive_spectra(g._h, C.byref(air._view(v)), C.byref(p), C.byref(im),
                                         C.c_void_p(pageable.ctypes.data), ref["n_out"]) == air.AIR_ERR_ARG
    pinned = torch.empty((sc.n_bands, ref["n_out"]), dtype=torch.float32, pin_memory=True)
    p0 = air.Params(16, 3, 0.3, 0, 0, -1, 0)
    assert L.air_render_adaptive_spectra(g._h, C.byref(air._view(v)), C.byref(p0), C.byref(im),
                                         C.c_void_p(pinned.data_ptr()), ref["n_out"]) == air.AIR_ERR_ARG
    small = torch.empty((sc.n_bands, 100), dtype=torch.float32, pin_memory=True)
    assert L.air_render_adaptive_spectra(g._h, C.byref(air._view(v)), C.byref(p), C.byref(im),
                                         C.c_void_p(small.data_ptr()), 100) == air.AIR_ERR_CAPACITY
    assert im.n_rays == ref["n_rays"]
