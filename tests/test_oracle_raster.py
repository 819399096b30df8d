"""Pins of the finest-level raster oracle (Section 2 step vi, bilinear
reading): hand-worked values on a mixed-level image, and closed forms."""
import json
import os

import numpy as np

from oracle import raster as R

GOLD = os.path.join(os.path.dirname(__file__), "golden", "raster_hand.json")


def test_hand_worked_mixed_level_image():
    g = json.load(open(GOLD))
    nodes = np.array(g["nodes"])
    lv, i, j, val = nodes[:, 0].astype(int), nodes[:, 1].astype(int), nodes[:, 2].astype(int), nodes[:, 3]
    for mode in ("bilinear", "nearest"):
        out = R.raster(lv, i, j, val, g["n0"], g["max_level"], mode)
        for key, want in g[mode].items():
            x, y = (int(s) for s in key.split(","))
            assert out[y, x] == want, (mode, key, out[y, x])


def _full_pyramid(n0, Lm, fn):
    lv, ii, jj, val = [], [], [], []
    for L in range(Lm + 1):
        nl = n0 << L
        y, x = np.meshgrid(np.arange(nl), np.arange(nl), indexing="ij")
        lv.append(np.full(nl * nl, L))
        ii.append(x.ravel())
        jj.append(y.ravel())
        val.append(fn(L, x.ravel(), y.ravel()))
    return [np.concatenate(a) for a in (lv, ii, jj, val)]


def test_finest_leaves_keep_their_values():
    rng = np.random.default_rng(1)
    vals = {}

    def fn(L, x, y):
        v = rng.normal(size=x.size)
        vals[L] = v.reshape(8 << L, 8 << L)
        return v
    lv, i, j, val = _full_pyramid(8, 2, fn)
    for mode in ("nearest", "bilinear"):
        np.testing.assert_array_equal(R.raster(lv, i, j, val, 8, 2, mode), vals[2])


def test_linear_image_is_reproduced_inside():
    """Base-level leaves only (no refinement): sampled at level-0 pixel
    centres, p = a + b u + c v is reproduced at every finest pixel whose
    four level-0 neighbours lie inside the image."""
    n0, Lm, a, b, c = 6, 2, 0.3, 1.7, -0.9
    y, x = np.meshgrid(np.arange(n0), np.arange(n0), indexing="ij")
    out = R.raster(np.zeros(n0 * n0, int), x.ravel(), y.ravel(), a + b * x.ravel() + c * y.ravel(),
                   n0, Lm)
    nf = n0 << Lm
    yy, xx = np.meshgrid(np.arange(nf), np.arange(nf), indexing="ij")
    u = (xx + 0.5) / 4 - 0.5
    v = (yy + 0.5) / 4 - 0.5
    inside = (u >= 0) & (u <= n0 - 1) & (v >= 0) & (v <= n0 - 1)
    np.testing.assert_allclose(out[inside], (a + b * u + c * v)[inside], rtol=0, atol=1e-13)
    # outside, clamping holds the edge value along the clamped axis
    np.testing.assert_allclose(out[0, :], out[1, :], rtol=0, atol=1e-13)


def test_constant_stays_constant_on_any_tree():
    rng = np.random.default_rng(3)
    n0, Lm = 4, 3
    lv, ii, jj = [0] * 16, list(np.tile(np.arange(4), 4)), list(np.repeat(np.arange(4), 4))
    frontier = list(zip(lv, ii, jj))
    for L in range(Lm):
        nxt = []
        for (l, i, j) in frontier:
            if rng.random() < 0.5:
                for dj in (0, 1):
                    for di in (0, 1):
                        nxt.append((l + 1, 2 * i + di, 2 * j + dj))
        lv += [n[0] for n in nxt]
        ii += [n[1] for n in nxt]
        jj += [n[2] for n in nxt]
        frontier = nxt
    for mode in ("nearest", "bilinear"):
        out = R.raster(np.array(lv), np.array(ii), np.array(jj), np.full(len(lv), 2.5), n0, Lm, mode)
        assert np.all(out == 2.5)
