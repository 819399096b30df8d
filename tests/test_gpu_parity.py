"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: every pixel value (column density N, intensity I_b) within
1e-5 relative of the oracle, plus an absolute floor of 1e-7 x the image
maximum for pixels whose value comes from a sliver of a cell (a grazing
chord, where FP32 ray geometry dominates). Integer results (the refinement
tree, pixel layout, step counts on axis views) are compared exactly."""
import math

import numpy as np
import pytest

import oracle
import paper_1010_5534_gb300 as air
import scenes
import test_oracle_camera as camera_pins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

RTOL = 1e-5
FLOOR = 1e-7


@pytest.fixture(scope="module", autouse=True)
def _built():
    air.build()


def close(gpu, orc, what, rtol=RTOL, floor=FLOOR, max_floor_frac=1e-3):
    """Element-wise |gpu - oracle| <= rtol |oracle| + floor max|oracle|.
    Returns how many values pass only thanks to the absolute floor (printed;
    at most max_floor_frac of them may)."""
    g = np.asarray(gpu, dtype=np.float64)
    o = np.asarray(orc, dtype=np.float64)
    assert g.shape == o.shape, (what, g.shape, o.shape)
    atol = floor * max(float(np.abs(o).max()) if o.size else 0.0, 1e-300)
    err = np.abs(g - o)
    bad = err > rtol * np.abs(o) + atol
    if bad.any():
        k = int(np.argmax(err / (rtol * np.abs(o) + atol)))
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} off (max |oracle| {np.abs(o).max():.4g}); "
                             f"worst at {k}: gpu {g.flat[k]!r} oracle {o.flat[k]!r} "
                             f"rel {err.flat[k] / max(abs(o.flat[k]), 1e-300):.3e}")
    n_floor = int((err > rtol * np.abs(o)).sum())
    print(f"[close] {what}: {g.size} values, {n_floor} within tolerance only by the floor")
    assert n_floor <= max_floor_frac * g.size + 1, (what, n_floor, g.size)
    return n_floor


def np_(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


# ------------------------------------------------------------------ scenes
@pytest.fixture(scope="module")
def wind():
    s = scenes.wind_shell_uniform(0)
    return s, air.Grid(s), oracle.Oracle(s)


@pytest.fixture(scope="module")
def cone4():
    s = scenes.cone_shock_amr(1, n_base=32, brick=8, levels=2, n_bands=4, e_lo=0.5, e_hi=10.0,
                              kappa0=0.4, thickness=0.08)
    return s, air.Grid(s), oracle.Oracle(s)


@pytest.fixture(scope="module")
def cone1():
    s = scenes.cone_shock_amr(2, n_base=32, brick=8, levels=2)
    return s, air.Grid(s), oracle.Oracle(s)


def fixed_pair(sc, g, o, view, res, **kw):
    r = g.render_fixed(view, res, **kw)
    f = o.fixed(view, res)
    return r, f


# ------------------------------------------------------------------ fixed images
@pytest.mark.parametrize("res", [128, 100])
def test_fixed_uniform_axis(wind, res):
    sc, g, o = wind
    v = scenes.axis_view("+z")
    r, f = fixed_pair(sc, g, o, v, res)
    assert r["n_out"] == res * res
    assert (np_(r["i"]) == f["i"]).all() and (np_(r["j"]) == f["j"]).all()
    close(np_(r["coldens"]), f["col"], "N")
    close(np_(r["intensity"])[0], f["inten"][:, 0], "I")
    # axis view: segment counts are exact
    assert r["n_steps"] == int(f["steps"].sum())
    flux = (f["inten"][:, 0] * (2.0 / res) ** 2).sum()
    assert np_(r["band_flux"])[0] == pytest.approx(flux, rel=RTOL)


def test_fixed_uniform_oblique(wind):
    sc, g, o = wind
    for v in scenes.random_views(4, 3):
        r, f = fixed_pair(sc, g, o, v, 61)
        close(np_(r["coldens"]), f["col"], "N")
        close(np_(r["intensity"])[0], f["inten"][:, 0], "I")
        # FP32 cell boundaries next to an edge or corner can add a sliver
        # segment that the exact line only touches: counts agree to 1e-3
        assert abs(r["n_steps"] - f["steps"].sum()) <= 1e-3 * f["steps"].sum() + 8


@pytest.mark.parametrize("fp64_level", [-1, 0, 99])
def test_fixed_amr_multiband(cone4, fp64_level):
    sc, g, o = cone4
    views = [scenes.axis_view("+z"), scenes.axis_view("-x")] + scenes.random_views(9, 2)
    for v in views:
        r, f = fixed_pair(sc, g, o, v, 77, fp64_level=fp64_level)
        close(np_(r["coldens"]), f["col"], f"N {v.dir}")
        I = np_(r["intensity"])
        for b in range(sc.n_bands):
            close(I[b], f["inten"][:, b], f"I[{b}] {v.dir}")
        pf = f["inten"].sum(axis=1)
        close(np_(r["p"]), pf, "p")


def test_axis_rays_with_and_without_column_tables(cone4):
    """Rays along a grid axis take their two fixed cells from a per-column
    table when the image plane's u and v are grid axes too, and from the FP64
    set-up otherwise (+z with the image plane turned 30 degrees about it).
    Both agree with the oracle, step counts exactly; and the table path gives
    the same bits as the batched kernel, which always takes the FP64 set-up."""
    sc, g, o = cone4
    c, s_ = math.cos(math.radians(30.0)), math.sin(math.radians(30.0))
    turned = scenes.View(dir=(0.0, 0.0, 1.0), up=(s_, c, 0.0))
    for v in (scenes.axis_view("+z"), turned):
        r, f = fixed_pair(sc, g, o, v, 77)
        close(np_(r["coldens"]), f["col"], f"N {v.up}")
        close(np_(r["intensity"])[0], f["inten"][:, 0], f"I {v.up}")
        assert r["n_steps"] == int(f["steps"].sum())
        _hybrid_check(g, o, v, 16, 3, 0.4)
    v = scenes.axis_view("+z")
    a = g.render_adaptive(v, 16, 3, 0.4)
    b = g.render_batch([v], 16, 3, 0.4)[0]
    for k in ("level", "i", "j", "coldens", "intensity"):
        assert (np_(a[k]) == np_(b[k])).all(), k


def test_fixed_image_missing_the_box(wind):
    sc, g, o = wind
    v = scenes.View(dir=(0, 0, 1), center=(5.0, 0.0, 0.0), half_extent=1.0)
    r = g.render_fixed(v, 16)
    assert float(np_(r["coldens"]).max()) == 0.0 and r["n_steps"] == 0
    assert float(np_(r["band_flux"])[0]) == 0.0


def test_fixed_res_one_and_face_aligned(wind):
    sc, g, o = wind
    for res in (1, 2, 32, 64):   # res 2, 32, 64: pixel centres on cell faces
        r, f = fixed_pair(sc, g, o, scenes.axis_view("+y"), res)
        close(np_(r["coldens"]), f["col"], f"N res {res}")
        close(np_(r["intensity"])[0], f["inten"][:, 0], f"I res {res}")


def test_face_aligned_rays_with_inexact_reciprocal_cell_size():
    """Box of width 10 with 32 cells: h = 5/16 is exact but 1/h = 3.2 is not.
    Pixel centres of a 16^2 image lie exactly on cell faces; the half-open rule
    must pick the higher cell exactly as the oracle's division does."""
    rng = np.random.default_rng(5)
    rho = np.exp(rng.normal(size=(32, 32, 32)))
    sc = scenes.uniform_from_array(rho, lo=(-5.0,) * 3, hi=(5.0,) * 3, kappa=0.05)
    g, o = air.Grid(sc), oracle.Oracle(sc)
    for axis in ("+x", "-y", "+z"):
        v = scenes.axis_view(axis, half_extent=5.0)
        for res in (16, 8):
            r, f = fixed_pair(sc, g, o, v, res)
            close(np_(r["coldens"]), f["col"], f"N {axis} {res}")
            close(np_(r["intensity"])[0], f["inten"][:, 0], f"I {axis} {res}")
            assert r["n_steps"] == int(f["steps"].sum())


@pytest.mark.parametrize("case", range(len(camera_pins.CASES)),
                         ids=[c[0] for c in camera_pins.CASES])
def test_camera_axes_on_gpu(case):
    """The hand-derived camera pins (image axis and sign of each world axis,
    the paper's face-on ring view among them) hold for the CUDA path too."""
    name, view, cond, expect = camera_pins.CASES[case]
    sc = scenes.uniform_from_array(camera_pins._field(cond), kappa=0.0)
    g = air.Grid(sc)
    r = g.render_fixed(view, camera_pins.RES)
    img = np_(r["intensity"])[0]
    lit = {(int(i), int(j)) for i, j, x in zip(np_(r["i"]), np_(r["j"]), img) if x > 0.0}
    assert lit == expect, name
    assert np.allclose(img[img > 0.0], 2.0, rtol=1e-6)
    g.close()


# ------------------------------------------------------------------ adaptive images
def nodes_of(r):
    return {k: np_(r[k]) for k in ("level", "i", "j", "is_leaf", "coldens", "p")} | \
        {"I": np_(r["intensity"])}


@pytest.mark.parametrize("xc", [0.2, 0.5, 0.8])
def test_air_uniform_matches_oracle(wind, xc):
    sc, g, o = wind
    v = scenes.axis_view("+z")
    r = g.render_adaptive(v, 16, 3, xc, include_interior=True)
    t = o.air(v, 16, 3, xc)
    n = nodes_of(r)
    assert r["n_rays"] == t["n_nodes"] and r["n_leaves"] == t["n_leaves"]
    assert r["n_sweeps"] == t["n_sweeps"]
    for k in ("level", "i", "j"):
        assert (n[k] == t[k]).all(), k
    assert (n["is_leaf"] == t["leaf"]).all()
    close(n["coldens"], t["col"], "N")
    close(n["I"][0], t["inten"][:, 0], "I")
    assert np_(r["band_flux"])[0] == pytest.approx(t["band_flux"][0], rel=RTOL)
    assert r["n_steps"] == t["n_steps"]


def _replay_check(g, o, v, n0, Lm, xc, **kw):
    r = g.render_adaptive(v, n0, Lm, xc, include_interior=True, **kw)
    n = nodes_of(r)
    rp = dict(level=n["level"], i=n["i"], j=n["j"], p_int=n["p"].astype(np.float64),
              p_col=n["coldens"].astype(np.float64))
    kw2 = {k: kw[k] for k in ("xi_norm", "refine_on") if k in kw}
    t = o.air(v, n0, Lm, xc, replay=rp, **kw2)
    assert t["n_nodes"] == r["n_rays"]
    for k in ("level", "i", "j"):
        assert (t[k] == n[k]).all(), k
    assert (t["leaf"] == n["is_leaf"]).all()
    return r


@pytest.mark.parametrize("refine_on,xi_norm", [(0, 0), (1, 0), (2, 1), (0, 1)])
def test_air_refinement_bit_exact_on_gpu_values(cone4, refine_on, xi_norm):
    """Fed the GPU's own FP32 pixel values, the oracle's scan/balance/refine
    loop reproduces the GPU quadtree exactly (node by node, in order)."""
    sc, g, o = cone4
    for v in (scenes.axis_view("+z"), scenes.random_views(5, 1)[0]):
        _replay_check(g, o, v, 12, 3, 0.3, refine_on=refine_on, xi_norm=xi_norm)


def _hybrid_check(g, o, v, n0, Lm, xc, capacity=None, **kw):
    """GPU tree against the oracle's tree from its own FP64 march. Every flag
    decision whose xi is farther from xi_crit than twice the first-order
    change that a 1e-5 relative change of the stencil values can cause is the
    oracle's own; the undecided rest take the GPU's values (orc_air_hybrid).
    The GPU tree must equal that tree node for node, and every node's values
    must match the oracle's own trace."""
    r = g.render_adaptive(v, n0, Lm, xc, include_interior=True, **kw)
    n = nodes_of(r)
    other = dict(level=n["level"], i=n["i"], j=n["j"], p_int=n["p"].astype(np.float64),
                 p_col=n["coldens"].astype(np.float64))
    kw2 = {k: kw[k] for k in ("xi_norm", "refine_on") if k in kw}
    t = o.air(v, n0, Lm, xc, other=other, rtol=RTOL, margin=2.0, capacity=capacity, **kw2)
    hy = t["hybrid"]
    print(f"[tree] {n0}^2 L{Lm} xi_crit {xc}: {t['n_nodes']} nodes, {hy['decisions']} decisions, "
          f"{hy['undecided']} undecided, {hy['taken_from_other']} of them resolved unlike the "
          f"oracle's own values, {hy['unresolved']} unresolvable")
    assert hy["unresolved"] == 0
    assert t["n_nodes"] == r["n_rays"], (t["n_nodes"], r["n_rays"])
    for k in ("level", "i", "j"):
        assert (t[k] == n[k]).all(), k
    assert (t["leaf"] == n["is_leaf"]).all()
    close(n["coldens"], t["col"], "N")
    for b in range(t["inten"].shape[1]):
        close(n["I"][b], t["inten"][:, b], f"I[{b}]")
    return r, t


def test_air_amr_matches_oracle_on_decided_nodes(cone1, cone4, wind):
    """Own FP64 march on the oracle side: the trees agree on every decided
    node, the undecided ones are counted."""
    sc, g, o = cone1
    _hybrid_check(g, o, scenes.axis_view("+z"), 32, 3, 0.5)
    _hybrid_check(g, o, scenes.random_views(7, 1)[0], 24, 3, 0.4)
    sc, g, o = cone4
    for v in (scenes.axis_view("-x"), scenes.random_views(11, 1)[0]):
        _hybrid_check(g, o, v, 16, 3, 0.3, refine_on=2)
    sc, g, o = wind
    for xc in (0.2, 0.5, 0.8):
        _hybrid_check(g, o, scenes.axis_view("+z"), 16, 3, xc)


def test_air_zero_threshold_equals_fixed_finest(cone4):
    sc, g, o = cone4
    v = scenes.axis_view("+z")
    r = g.render_adaptive(v, 8, 3, 0.0)
    f = g.render_fixed(v, 64)
    lv, i, j = np_(r["level"]), np_(r["i"]), np_(r["j"])
    assert (lv == 3).all() and r["n_out"] == 64 * 64
    order = np.argsort(j * 64 + i)
    assert (np_(r["coldens"])[order] == np_(f["coldens"])).all()
    assert (np_(r["intensity"])[:, order] == np_(f["intensity"])).all()


def test_air_invariants_and_threshold_extremes(cone1):
    sc, g, o = cone1
    v = scenes.axis_view("+z")
    r = g.render_adaptive(v, 16, 4, 1.01)
    assert r["n_rays"] == 256 and r["n_sweeps"] == 0 and r["n_leaves"] == 256
    for xc in (0.5, 0.1):
        r = g.render_adaptive(v, 16, 4, xc)
        nref = (r["n_rays"] - 256) // 4
        assert r["n_rays"] == 256 + 4 * nref and r["n_leaves"] == 256 + 3 * nref
        lv, i, j = np_(r["level"]), np_(r["i"]), np_(r["j"])
        nf = 16 << 4
        R = np.full((nf, nf), -1)
        for L, a, b in zip(lv, i, j):
            s = 1 << (4 - L)
            assert (R[b * s:(b + 1) * s, a * s:(a + 1) * s] == -1).all()
            R[b * s:(b + 1) * s, a * s:(a + 1) * s] = L
        assert (R >= 0).all()
        for dj, di in ((0, 1), (1, 0), (1, 1), (1, -1)):
            A = R[max(dj, 0):nf + min(dj, 0), max(di, 0):nf + min(di, 0)]
            B = R[max(-dj, 0):nf + min(-dj, 0), max(-di, 0):nf + min(-di, 0)]
            assert np.abs(A - B).max() <= 1


def test_air_edge_sizes(wind):
    sc, g, o = wind
    v = scenes.axis_view("+z")
    for n0, Lm, xc in ((1, 0, 0.5), (1, 4, 0.2), (3, 3, 0.4), (5, 2, 0.0)):
        r = g.render_adaptive(v, n0, Lm, xc, include_interior=True)
        t = o.air(v, n0, Lm, xc)
        n = nodes_of(r)
        assert r["n_rays"] == t["n_nodes"], (n0, Lm)
        for k in ("level", "i", "j"):
            assert (n[k] == t[k]).all()
        close(n["I"][0], t["inten"][:, 0], "I")


def test_host_and_device_outputs_agree(cone4):
    sc, g, o = cone4
    v = scenes.random_views(2, 1)[0]
    d = g.render_adaptive(v, 16, 2, 0.4, mem="device")
    h = g.render_adaptive(v, 16, 2, 0.4, mem="host")
    for k in ("level", "i", "j", "coldens", "intensity", "p", "band_flux"):
        assert (np_(d[k]) == np_(h[k])).all(), k
    fd = g.render_fixed(v, 33, mem="device")
    fh = g.render_fixed(v, 33, mem="host")
    for k in ("coldens", "intensity", "p"):
        assert (np_(fd[k]) == np_(fh[k])).all(), k


def test_capacity_retry_and_profile(cone1):
    sc, g, o = cone1
    v = scenes.axis_view("+z")
    g.profile(True)
    r1 = g.render_adaptive(v, 16, 3, 0.3, capacity=10)     # too small -> retry inside
    r2 = g.render_adaptive(v, 16, 3, 0.3)
    assert r1["n_out"] == r2["n_out"]
    assert (np_(r1["coldens"]) == np_(r2["coldens"])).all()
    prof = g.profile_read()
    assert prof["march"][1] > 0 and prof["march"][0] > 0.0
    assert prof["scan"][1] > 0 and prof["output"][1] > 0
    g.profile(False)


def test_bad_arguments(wind):
    sc, g, o = wind
    v = scenes.axis_view("+z")
    with pytest.raises(air.AirError) as e:
        g.render_adaptive(v, 0, 3, 0.5)
    assert e.value.status == air.AIR_ERR_ARG
    with pytest.raises(air.AirError):
        g.render_adaptive(v, 16, 3, -1.0)
    with pytest.raises(air.AirError):
        g.render_adaptive(scenes.View(dir=(0, 1, 0), up=(0, 2, 0)), 16, 3, 0.5)
    with pytest.raises(air.AirError):
        g.render_fixed(v, 0)
    bad = scenes.wind_shell_uniform(0, n=8)
    bad.rho[1, 2, 3] = -1.0
    with pytest.raises(air.AirError) as e:
        air.Grid(bad)
    assert e.value.status == air.AIR_ERR_ARG
    amr = scenes.cone_shock_amr(0, n_base=16, brick=4, levels=1)
    amr.brick_level = amr.brick_level[:-1].copy()   # hole in the tiling
    amr.brick_origin = amr.brick_origin[:-1].copy()
    amr.rho = amr.rho[:-1].copy()
    amr.temp = amr.temp[:-1].copy()
    with pytest.raises(air.AirError):
        air.Grid(amr)
    # the library stays usable after errors
    r = g.render_fixed(v, 8)
    assert r["n_out"] == 64


# ------------------------------------------------------------------ full size (bench config)
@pytest.fixture(scope="module")
def cone_full():
    sc = scenes.cone_shock_amr(0)
    return sc, air.Grid(sc), oracle.Oracle(sc)


def test_cone_full_size_sampled(cone_full):
    """The 128^3-base, 16^3-brick, 3-level cone-shock grid at the benchmark's
    launch configuration (256^2 base image, max level 4, xi_crit 0.5): sampled
    leaves against the oracle ray by ray, the tree invariants, and the band
    flux within the metric's 1e-4 of the fixed 4096^2 image."""
    sc, g, o = cone_full
    v = scenes.axis_view("+z")
    r = g.render_adaptive(v, 256, 4, 0.5)
    nref = (r["n_rays"] - 65536) // 4
    assert r["n_rays"] == 65536 + 4 * nref and r["n_leaves"] == 65536 + 3 * nref
    lv, i, j = np_(r["level"]), np_(r["i"]), np_(r["j"])
    rng = np.random.default_rng(0)
    pick = rng.choice(len(lv), size=4000, replace=False)
    col, inten, _ = o.trace(v, 256, lv[pick], i[pick], j[pick])
    close(np_(r["coldens"])[pick], col, "N")
    close(np_(r["intensity"])[0][pick], inten[:, 0], "I")
    f = g.render_fixed(v, 4096, fields=("band_flux",))
    err = abs(np_(r["band_flux"])[0] - np_(f["band_flux"])[0]) / np_(f["band_flux"])[0]
    print(f"[flux] AIR vs fixed 4096^2: relative error {err:.3e}")
    assert err <= 1e-4


def test_cone_full_size_tree_replay(cone_full):
    """The bench image's whole quadtree (7.7 M nodes, 8 sweeps, the multi-block
    scan and emit kernels at full width): the oracle's sweep loop fed the GPU's
    FP32 pixel values reproduces it node for node (level, i, j, order, leaf)."""
    sc, g, o = cone_full
    v = scenes.axis_view("+z")
    r = g.render_adaptive(v, 256, 4, 0.5, include_interior=True,
                          fields=("level", "i", "j", "is_leaf", "coldens", "p"))
    n = {k: np_(r[k]) for k in ("level", "i", "j", "is_leaf", "coldens", "p")}
    rp = dict(level=n["level"], i=n["i"], j=n["j"], p_int=n["p"].astype(np.float64),
              p_col=n["coldens"].astype(np.float64))
    t = o.air(v, 256, 4, 0.5, replay=rp, capacity=int(r["n_rays"]))
    assert t["n_nodes"] == r["n_rays"] and t["n_sweeps"] == r["n_sweeps"]
    for k in ("level", "i", "j"):
        assert (t[k] == n[k]).all(), k
    assert (t["leaf"] == n["is_leaf"]).all()


def test_cone_full_size_own_march_tree(cone_full):
    """The same image against the oracle's own FP64 march of all 7.7 M rays:
    identical tree on every decided node (undecided ones counted), and every
    pixel value within tolerance."""
    sc, g, o = cone_full
    r, t = _hybrid_check(g, o, scenes.axis_view("+z"), 256, 4, 0.5, capacity=8_200_000)
    assert r["n_steps"] == t["n_steps"]


def test_reused_output_arrays(cone4):
    """render_adaptive(out=...) writes the image into caller-held arrays, call
    after call, with the bits of a fresh call; arrays that are too small fail
    with AIR_ERR_CAPACITY."""
    sc, g, o = cone4
    v = scenes.random_views(5, 1)[0]
    ref = g.render_adaptive(v, 16, 2, 0.4)
    n = ref["n_out"]
    fields = ("level", "i", "j", "coldens", "intensity", "band_flux")
    for mem in ("device", "host"):
        buf = g.alloc_image(n + 7, mem, fields)
        for rep in range(2):
            r = g.render_adaptive(v, 16, 2, 0.4, mem=mem, out=buf)
            assert r["n_out"] == n
            for k in fields:
                assert (np_(r[k]) == np_(ref[k])).all(), (mem, rep, k)
            assert r["intensity"].data_ptr() == buf["intensity"].data_ptr()
    small = g.alloc_image(max(n // 2, 1), "device", fields)
    with pytest.raises(air.AirError) as e:
        g.render_adaptive(v, 16, 2, 0.4, out=small)
    assert e.value.status == air.AIR_ERR_CAPACITY
    with pytest.raises(ValueError):
        g.render_adaptive(v, 16, 2, 0.4, mem="host", out=small)


def test_pageable_host_outputs_use_staging(cone4):
    """Host outputs in pageable memory go through device staging and copies,
    as page-locked ones do. Same bits as device outputs."""
    import ctypes as C
    sc, g, o = cone4
    v = scenes.random_views(3, 1)[0]
    d = g.render_adaptive(v, 16, 2, 0.4, mem="device")
    n = d["n_out"]
    arr = dict(level=np.zeros(n, np.int32), i=np.zeros(n, np.int32), j=np.zeros(n, np.int32),
               is_leaf=np.zeros(n, np.uint8), coldens=np.zeros(n, np.float32),
               p=np.zeros(n, np.float32), intensity=np.zeros((sc.n_bands, n), np.float32),
               band_flux=np.zeros(sc.n_bands, np.float64))
    im = air.Image()
    im.mem = air.AIR_HOST
    im.capacity = n
    for k, a in arr.items():
        setattr(im, k, a.ctypes.data)
    p = air.Params(16, 2, 0.4, 0, 0, -1, 0)
    assert air.lib().air_render_adaptive(g._h, C.byref(air._view(v)), C.byref(p), C.byref(im)) == air.AIR_OK
    for k in ("level", "i", "j", "coldens", "p", "intensity", "band_flux"):
        assert (arr[k] == np_(d[k])).all(), k
