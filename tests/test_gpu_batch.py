"""Batched adaptive images (one cooperative persistent kernel for every sweep of
every view, launched through a CUDA graph): each view must equal its
single-view render exactly -- same pixels, same order, same values -- whatever
the band split, with or without the graph, to host or device memory. The
single-view path is itself checked against the FP64 oracle in
test_gpu_parity.py; two views are re-checked here against the oracle fed the
batch's own pixel values. A grid-barrier wait that runs out returns
AIR_ERR_TIMEOUT and leaves the GPU usable."""
import numpy as np
import pytest

import oracle
import paper_1010_5534_gb300 as air
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

KEYS = ("level", "i", "j", "is_leaf", "coldens", "intensity", "p")


def np_(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


@pytest.fixture(scope="module")
def cone():
    air.build()
    s = scenes.cone_shock_amr(4, n_base=32, brick=8, levels=2, n_bands=5, e_lo=0.5, e_hi=10.0,
                              kappa0=0.4, thickness=0.08)
    return s, air.Grid(s)


def views5():
    return [scenes.axis_view("+z"), scenes.axis_view("-x")] + scenes.random_views(21, 3)


def same(a, b, what):
    for k in KEYS:
        x, y = np_(a[k]), np_(b[k])
        assert x.shape == y.shape and (x == y).all(), (what, k)
    for k in ("n_out", "n_leaves", "n_rays", "n_sweeps", "n_steps"):
        assert a[k] == b[k], (what, k, a[k], b[k])
    np.testing.assert_allclose(np_(a["band_flux"]), np_(b["band_flux"]), rtol=1e-12)


@pytest.mark.parametrize("bpt", [0, 1, 2, 4])
def test_batch_equals_single_views(cone, bpt):
    sc, g = cone
    vs = views5()
    singles = [g.render_adaptive(v, 12, 3, 0.3, include_interior=True) for v in vs]
    batch = g.render_batch(vs, 12, 3, 0.3, include_interior=True, bands_per_thread=bpt)
    for k, (a, b) in enumerate(zip(batch, singles)):
        same(a, b, f"view {k} bpt {bpt}")


def test_batch_leaves_graph_direct_and_host(cone):
    sc, g = cone
    vs = views5()
    singles = [g.render_adaptive(v, 16, 2, 0.5, refine_on=2, xi_norm=1) for v in vs]
    for use_graph in (True, False):
        for rep in range(2):          # a second call replays the captured graph
            b = g.render_batch(vs, 16, 2, 0.5, refine_on=2, xi_norm=1, use_graph=use_graph)
            for k in range(len(vs)):
                same(b[k], singles[k], f"graph {use_graph} rep {rep} view {k}")
    h = g.render_batch(vs, 16, 2, 0.5, refine_on=2, xi_norm=1, mem="host")
    for k in range(len(vs)):
        same(h[k], singles[k], f"host view {k}")


def test_batch_matches_oracle_replay(cone):
    sc, g = cone
    o = oracle.Oracle(sc)
    vs = views5()[:2]
    b = g.render_batch(vs, 12, 3, 0.3, include_interior=True)
    for v, r in zip(vs, b):
        rp = dict(level=np_(r["level"]), i=np_(r["i"]), j=np_(r["j"]),
                  p_int=np_(r["p"]).astype(np.float64), p_col=np_(r["coldens"]).astype(np.float64))
        t = o.air(v, 12, 3, 0.3, replay=rp)
        for k in ("level", "i", "j"):
            assert (t[k] == np_(r[k])).all()
        # values against the oracle's own march
        col, inten, _ = o.trace(v, 12, np_(r["level"]), np_(r["i"]), np_(r["j"]))
        I = np_(r["intensity"]).astype(np.float64)
        for bnd in range(sc.n_bands):
            err = np.abs(I[bnd] - inten[:, bnd])
            assert (err <= 1e-5 * np.abs(inten[:, bnd]) + 1e-7 * np.abs(inten[:, bnd]).max()).all()


def test_batch_growth_and_many_views(cone):
    sc, g = cone
    vs = scenes.random_views(33, 40)
    b = g.render_batch(vs, 8, 3, 0.2)
    for k in (0, 17, 39):
        s1 = g.render_adaptive(vs[k], 8, 3, 0.2)
        same(b[k], s1, f"view {k}")


def test_batch_bounded_wait_returns_timeout(cone):
    sc, g = cone
    vs = views5()[:2]
    with pytest.raises(air.AirError) as e:
        g.render_batch(vs, 8, 2, 0.5, test_stall_barrier=True, wait_timeout_ms=50.0,
                       use_graph=False)
    assert e.value.status == air.AIR_ERR_TIMEOUT
    # the context stays usable
    b = g.render_batch(vs, 8, 2, 0.5)
    s = g.render_adaptive(vs[1], 8, 2, 0.5)
    same(b[1], s, "after timeout")


def test_batch_equals_single_views_one_band():
    """One-band grid: a single-view render of a face-on view runs the compiled
    one-axis march kernel, the batched kernel the general form with its
    run-time choice of the one-axis loop; the bits must agree."""
    s = scenes.cone_shock_amr(5, n_base=32, brick=8, levels=2, thickness=0.08)
    g = air.Grid(s)
    vs = [scenes.axis_view(a) for a in ("+z", "-x", "+y")] + scenes.random_views(22, 1)
    singles = [g.render_adaptive(v, 16, 3, 0.3, include_interior=True) for v in vs]
    batch = g.render_batch(vs, 16, 3, 0.3, include_interior=True)
    for k, (a, b) in enumerate(zip(batch, singles)):
        same(a, b, f"one-band view {k}")
    for v in vs[:3]:   # fixed images too (one-axis kernel) against the same rays in a batch base image
        f = g.render_fixed(v, 16)
        b = g.render_batch([v], 16, 0, 0.3, include_interior=True)[0]
        assert (np_(f["coldens"]) == np_(b["coldens"])).all()
        assert (np_(f["intensity"]) == np_(b["intensity"])).all()
    g.close()
