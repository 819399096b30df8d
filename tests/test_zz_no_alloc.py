"""air_band_flux_static: the band flux of an image already on the device,
for callers that cannot allocate (a render loop that must not stall the GPU
on cudaFree, a plugin whose host owns the device memory pool). Its only scratch
is a fixed array inside the library. Checked against the band flux returned by
the regular render entry points, on two calls in a row through the C ABI.

Collected last on purpose (file name), so that a stop-at-first-failure run has
already run every other test; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

import paper_1010_5534_gb300 as air
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

RTOL = 1e-5


def _call(I, n, area0, level, leaf, out):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return air.lib().air_band_flux_static(
        C.c_void_p(I.data_ptr()), int(I.stride(0)), int(I.shape[0]),
        C.c_void_p(level.data_ptr()) if level is not None else None,
        C.c_void_p(leaf.data_ptr()) if leaf is not None else None, int(n), float(area0),
        C.c_void_p(out.data_ptr()), stream)


def test_static_flux_matches_render_twice():
    air.build()
    sc = scenes.cone_shock_amr(1, n_base=32, brick=8, levels=2, n_bands=3, e_lo=0.5,
                               kappa0=0.4, thickness=0.08)
    g = air.Grid(sc)
    v = scenes.random_views(5, 1)[0]
    n0 = 16
    area0 = (2.0 * v.half_extent / n0) ** 2
    out = torch.empty(sc.n_bands, dtype=torch.float64, device="cuda")
    # adaptive image with interior nodes: only leaves count
    r = g.render_adaptive(v, n0, 3, 0.3, include_interior=True)
    ref = r["band_flux"].cpu().numpy()
    assert (ref > 0).all()
    for _ in range(2):
        out.fill_(float("nan"))
        st = _call(r["intensity"], r["n_out"], area0, r["level"], r["is_leaf"], out)
        assert st == air.AIR_OK, air.lib().air_last_error()
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL, atol=0)
    # fixed image: every entry a level-0 pixel
    res = 48
    f = g.render_fixed(v, res)
    ref_f = f["band_flux"].cpu().numpy()
    for _ in range(2):
        out.fill_(float("nan"))
        st = _call(f["intensity"], f["n_out"], (2.0 * v.half_extent / res) ** 2, None, None, out)
        assert st == air.AIR_OK, air.lib().air_last_error()
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref_f, rtol=RTOL, atol=0)
    g.close()


def test_static_flux_rejects_sizes_beyond_its_scratch():
    air.build()
    I = torch.zeros((65, 8), dtype=torch.float32, device="cuda")
    out = torch.empty(65, dtype=torch.float64, device="cuda")
    assert _call(I, 8, 1.0, None, None, out) == air.AIR_ERR_ARG
    assert b"static scratch limit" in air.lib().air_last_error()
    J = torch.zeros((2, 8), dtype=torch.float32, device="cuda")
    st = air.lib().air_band_flux_static(C.c_void_p(J.data_ptr()), 1 << 32, 2, None, None, 1 << 31,
                                        1.0, C.c_void_p(out.data_ptr()), None)
    assert st == air.AIR_ERR_ARG
    # n valid, only the stride out of range: (n_bands - 1) * stride overflows int64
    st = air.lib().air_band_flux_static(C.c_void_p(J.data_ptr()), 1 << 62, 3, None, None, 8,
                                        1.0, C.c_void_p(out.data_ptr()), None)
    assert st == air.AIR_ERR_ARG
    assert b"overflows" in air.lib().air_last_error()
    host = np.zeros((2, 8), dtype=np.float32)
    st = air.lib().air_band_flux_static(C.c_void_p(host.ctypes.data), 8, 2, None, None, 8, 1.0,
                                        C.c_void_p(out.data_ptr()), None)
    assert st == air.AIR_ERR_ARG


def test_static_flux_levels_up_to_the_render_maximum():
    """Levels 0..20 (every level a render can produce) scale by exactly 4^-L;
    a counted level outside that range turns the flux into NaN instead of a
    silently wrong power of two."""
    air.build()
    n = 21 * 40
    g = torch.Generator().manual_seed(3)
    I = torch.rand((2, n), generator=g, dtype=torch.float32).cuda()
    lev = torch.arange(n, dtype=torch.int32).remainder(21).cuda()
    leaf = torch.ones(n, dtype=torch.uint8).cuda()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    assert _call(I, n, 0.75, lev, leaf, out) == air.AIR_OK
    torch.cuda.synchronize()
    ref = (I.cpu().double().numpy() * 0.75 * 4.0 ** -lev.cpu().double().numpy()).sum(axis=1)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0)
    for bad in (21, -1):
        lev2 = lev.clone()
        lev2[7] = bad
        assert _call(I, n, 0.75, lev2, leaf, out) == air.AIR_OK
        torch.cuda.synchronize()
        assert np.isnan(out.cpu().numpy()).all(), bad
        leaf2 = leaf.clone()
        leaf2[7] = 0  # not counted: the bad level is ignored
        assert _call(I, n, 0.75, lev2, leaf2, out) == air.AIR_OK
        torch.cuda.synchronize()
        assert np.isfinite(out.cpu().numpy()).all(), bad


def test_static_flux_binding_checks_layout():
    air.build()
    I = torch.zeros((2, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        air.band_flux_static(I.double(), 8, 1.0)
    with pytest.raises(ValueError):
        air.band_flux_static(I.t().contiguous().t(), 8, 1.0)
    with pytest.raises(ValueError):
        air.band_flux_static(I, 9, 1.0)
    with pytest.raises(ValueError):
        air.band_flux_static(I, 8, 1.0, level=torch.zeros(8, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        air.band_flux_static(I, 8, 1.0, is_leaf=torch.ones(4, dtype=torch.uint8, device="cuda"))
    out = air.band_flux_static(I, 8, 1.0, level=torch.zeros(8, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == 0.0).all()
