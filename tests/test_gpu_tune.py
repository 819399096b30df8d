"""Autotuner: it returns valid knob values, and every knob setting gives
bitwise-identical images (the knobs only change how work maps to threads)."""
import numpy as np
import pytest

import paper_1010_5534_gb300 as air
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

KEYS = ("level", "i", "j", "coldens", "intensity", "p")


def np_(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def grid():
    air.build()
    s = scenes.cone_shock_amr(8, n_base=32, brick=8, levels=2, n_bands=6, e_lo=0.5, kappa0=0.4,
                              thickness=0.08)
    return s, air.Grid(s)


def test_autotune_picks_valid_knobs(grid):
    s, g = grid
    v = scenes.random_views(2, 1)[0]
    t = g.autotune(v, 16, 3, 0.3, n_views_batch=3)
    assert t["tile_w"] in (4, 8, 16, 32)
    assert t["bands_per_thread"] in (1, 2, 4, 8)
    assert t["batch_bands_per_thread"] in (1, 2, 4, 8)
    assert t["batch_blocks_per_sm"] in (0, 1, 2)
    assert t["trials"] >= 4 + 4 + 12 and all(x > 0 for x in t["best_ms"])


def test_every_knob_setting_gives_the_same_images(grid):
    s, g = grid
    v = scenes.random_views(3, 1)[0]
    g.set_tuning()
    ref_f = g.render_fixed(v, 45)
    ref_a = g.render_adaptive(v, 16, 3, 0.3)
    ref_b = g.render_batch([v, scenes.axis_view("+z")], 16, 3, 0.3)
    for tw, bpt, bbpt, per in ((4, 1, 1, 1), (16, 2, 2, 2), (32, 4, 4, 0), (1, 8, 8, 1)):
        g.set_tuning(tile_w=tw, bands_per_thread=bpt, batch_bands_per_thread=bbpt,
                     batch_blocks_per_sm=per)
        f = g.render_fixed(v, 45)
        a = g.render_adaptive(v, 16, 3, 0.3)
        b = g.render_batch([v, scenes.axis_view("+z")], 16, 3, 0.3)
        for k in KEYS:
            assert (np_(f[k]) == np_(ref_f[k])).all(), (tw, k)
            assert (np_(a[k]) == np_(ref_a[k])).all(), (bpt, k)
            for x, y in zip(b, ref_b):
                assert (np_(x[k]) == np_(y[k])).all(), (bbpt, per, k)
    g.set_tuning()
    with pytest.raises(air.AirError):
        g.set_tuning(tile_w=3)
