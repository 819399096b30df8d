"""The paper's test calculation (Section 3, Eq. 3, Table 1) on the oracle: a hot
ring on a 4^3-block, 8^3-cell, 4-level grid, seen face-on; AIR with a 32^2 base
and 4 levels against the fixed 512^2 image. The synthetic emission table stands
in for MEKAL, so absolute fluxes are not comparable; what Table 1 fixes is the
shape: the fixed image is exact ("~0"), AIR's pixel counts are a small fraction
of 512^2 and of the order of the table's, and AIR's flux error is small."""
import json
import os

import numpy as np
import pytest

import oracle
import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ring():
    s = scenes.ring_amr()
    return s, oracle.Oracle(s)


def _exact_flux(s):
    tab = s.lambda_table[0].astype(np.float64)
    nt = tab.size
    hf = (s.hi[0] - s.lo[0]) / (s.n[0] << s.max_level)
    ex = 0.0
    for b in range(len(s.brick_level)):
        T = s.temp[b].astype(np.float64)
        x = np.clip((np.log10(T) - s.logT_lo) / (s.logT_hi - s.logT_lo) * (nt - 1), 0, nt - 1)
        k = np.minimum(np.floor(x).astype(int), nt - 2)
        w = x - k
        lam = (1 - w) * tab[k] + w * tab[k + 1]
        vol = (hf * (1 << (s.max_level - s.brick_level[b]))) ** 3
        ex += (s.rho[b].astype(np.float64) ** 2 * lam).sum() * vol
    return ex


def test_ring_grid_is_the_papers_layout(ring):
    s, _ = ring
    assert s.n == (32, 32, 32) and s.brick == 8 and s.max_level == 4
    assert (s.n[0] << s.max_level) == 512
    assert set(np.unique(s.brick_level)) == {0, 1, 2, 3, 4}


def test_table1_shape(ring):
    s, o = ring
    g = json.load(open(os.path.join(GOLD, "table1_counts.json")))
    v = scenes.ring_view()
    ex = _exact_flux(s)
    f = o.fixed(v, 512)
    A = (2 * v.half_extent / 512) ** 2
    assert abs(ex - f["inten"][:, 0].sum() * A) / ex < 1e-12          # "Fixed: ~0"
    for row in g["air"]:
        t = o.air(v, g["base_res"], g["levels"], row["xi_crit"])
        err = abs(ex - t["band_flux"][0]) / ex
        assert err < 1e-3
        assert 0.5 * row["pixels"] < t["n_nodes"] < 1.5 * row["pixels"], (row, t["n_nodes"])
        assert t["n_nodes"] < g["fixed_pixels"] / 6
