"""Parity at scale, through the C ABI against the FP64 oracle.

1. A grid whose finest level lies below the dense brick map: a 64^3 base of
   8^3 bricks refined six levels around small clumps has 512 x 8^6 > 2^24
   finest brick positions, so the map stops at level 5 and level-6 bricks are
   reached through the brick octree.
2. The large clumps-and-cones configuration at full size (512^3 base of 32^3
   bricks, 5 refinement levels, two shock cones, 200 clumps, 32 bands, base
   image 1024^2, max level 3): sampled leaves of the adaptive image against
   the oracle's rays for the same nodes.

Same tolerance as the other parity tests: 1e-5 relative plus an absolute
floor of 1e-7 x the largest oracle value."""
import os

import numpy as np
import pytest

import oracle
import paper_1010_5534_gb300 as air
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

RTOL = 1e-5
FLOOR = 1e-7


def close(gpu, orc, what):
    g = np.asarray(gpu, dtype=np.float64)
    o = np.asarray(orc, dtype=np.float64)
    atol = FLOOR * max(float(np.abs(o).max()) if o.size else 0.0, 1e-300)
    err = np.abs(g - o)
    bad = err > RTOL * np.abs(o) + atol
    if bad.any():
        k = int(np.argmax(err / (RTOL * np.abs(o) + atol)))
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} off; worst at {k}: gpu "
                             f"{g.flat[k]!r} oracle {o.flat[k]!r}")


def np_(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


@pytest.fixture(scope="module", autouse=True)
def _built():
    air.build()


def _centre(sc, b):
    hf = (sc.hi[0] - sc.lo[0]) / sc.finest_n[0]
    S = sc.brick << (sc.max_level - int(sc.brick_level[b]))
    return tuple(sc.lo[a] + (float(sc.brick_origin[b, a]) + 0.5 * S) * hf for a in range(3))


def test_octree_below_the_brick_map():
    sc = scenes.clumps_cones_amr(3, n_base=64, brick=8, levels=6, n_clumps=4,
                                 r_range=(0.004, 0.01), n_bands=2)
    assert (64 // 8) ** 3 * 8 ** 6 > 1 << 24          # the map stops above level 6
    deep = np.nonzero(sc.brick_level == 6)[0]
    assert len(deep) > 0
    g, o = air.Grid(sc), oracle.Oracle(sc)
    c = _centre(sc, int(deep[len(deep) // 2]))
    views = [scenes.View(dir=(0.0, 0.0, 1.0), center=c, half_extent=0.012),
             scenes.View(dir=(0.0, -1.0, 0.0), up=(0.0, 0.0, 1.0), center=c, half_extent=0.012)]
    rv = scenes.random_views(8, 1)[0]
    views.append(scenes.View(dir=rv.dir, up=rv.up, center=c, half_extent=0.012))
    for k, v in enumerate(views):
        r = g.render_fixed(v, 40)
        col, inten, steps = o.trace(v, 40, np.zeros(1600), np.tile(np.arange(40), 40),
                                    np.repeat(np.arange(40), 40))
        close(np_(r["coldens"]), col, f"N view {k}")
        I = np_(r["intensity"])
        for b in range(sc.n_bands):
            close(I[b], inten[:, b], f"I[{b}] view {k}")
        if k < 2:   # face-on: segment counts are exact
            assert r["n_steps"] == int(steps.sum())
    # the image crosses level-6 bricks: its rays take many more steps than the
    # 64 base cells across the box
    assert int(steps.max()) > 200
    g.close()


def _memory_ok(host_gb, dev_gb):
    try:
        host = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2 ** 30
    except (ValueError, OSError):
        host = 0.0
    dev = torch.cuda.get_device_properties(0).total_memory / 2 ** 30
    return host >= host_gb and dev >= dev_gb


@pytest.fixture(scope="module")
def large():
    if not _memory_ok(64, 40):
        pytest.skip("the full-size scene needs 64 GiB of host and 40 GiB of device memory")
    sc = scenes.clumps_cones_amr(0)
    g = air.Grid(sc)
    yield sc, g
    g.close()


@pytest.mark.parametrize("which", ["+z", "oblique"])
def test_large_amr_sampled_leaves_match_oracle(large, which):
    sc, g = large
    assert sc.n_bands == 32 and sc.max_level == 5 and int(sc.brick_level.max()) == 5
    v = scenes.axis_view("+z") if which == "+z" else scenes.random_views(11, 1)[0]
    r = g.render_adaptive(v, 1024, 3, 0.5)
    lv, ii, jj = np_(r["level"]), np_(r["i"]), np_(r["j"])
    n = len(lv)
    assert n == r["n_leaves"] and int(lv.max()) == 3
    rng = np.random.default_rng(5)
    pick = np.concatenate([rng.choice(n, 1000, replace=False),
                           rng.choice(np.nonzero(lv == 3)[0], 500, replace=False)])
    o = oracle.Oracle(sc)
    col, inten, steps = o.trace(v, 1024, lv[pick], ii[pick], jj[pick])
    close(np_(r["coldens"])[pick], col, "N")
    I = np_(r["intensity"])
    for b in range(sc.n_bands):
        close(I[b][pick], inten[:, b], f"I[{b}]")
