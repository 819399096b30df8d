"""GPU on the paper's ring problem (Section 3): the adaptive images at the three
thresholds of Table 1 are the oracle's trees node for node, with pixel values
within the parity tolerance, and the fixed 512^2 image is exact."""
import numpy as np
import pytest

import oracle
import paper_1010_5534_gb300 as air
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_ring_trees_match_oracle():
    air.build()
    s = scenes.ring_amr()
    g = air.Grid(s)
    o = oracle.Oracle(s)
    v = scenes.ring_view()
    for xc in (0.2, 0.5, 0.8):
        r = g.render_adaptive(v, 32, 4, xc, include_interior=True)
        t = o.air(v, 32, 4, xc)
        assert r["n_rays"] == t["n_nodes"], xc
        for k in ("level", "i", "j"):
            assert (r[k].cpu().numpy() == t[k]).all()
        I = r["intensity"][0].cpu().numpy().astype(np.float64)
        ref = t["inten"][:, 0]
        assert (np.abs(I - ref) <= 1e-5 * np.abs(ref) + 1e-7 * np.abs(ref).max()).all()
    f = g.render_fixed(v, 512)
    fo = o.fixed(v, 512)
    np.testing.assert_allclose(float(f["band_flux"][0]),
                               (fo["inten"][:, 0] * (10 / 512) ** 2).sum(), rtol=1e-6)
