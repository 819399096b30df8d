"""Learned refinement-depth proposal. Whatever the network proposes, the image
must be exactly plain AIR's (the paper's criterion, evaluated on every traced
pixel, decides); the labels it is trained on must be the depths of the
oracle's own tree; and a trained network must trace the image in fewer march
waves than plain AIR's sweep-by-sweep tracing."""
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
N0, LM, XC = 16, 3, 0.3


def np_(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


@pytest.fixture(scope="module")
def setup():
    air.build()
    s = scenes.cone_shock_amr(6, n_base=32, brick=8, levels=2, n_bands=2, e_lo=0.5,
                              kappa0=0.4, thickness=0.08)
    g = air.Grid(s)
    train_views = scenes.random_views(40, 24) + [scenes.axis_view("+z"), scenes.axis_view("+y")]
    xs, ys = [], []
    for v in train_views:
        x, y = g.learn_samples(v, N0, LM, XC)
        xs.append(x)
        ys.append(y)
    X = torch.cat(xs)
    Y = torch.cat(ys)
    net = air.MLP(scenes.mlp_init(1, scale=1.0))
    hist = net.train(X, Y, batch=512, epochs=30, lr=3e-3)
    return s, g, net, hist


def same(a, b, what):
    for k in KEYS:
        x, y = np_(a[k]), np_(b[k])
        assert x.shape == y.shape and (x == y).all(), (what, k)
    for k in ("n_out", "n_leaves", "n_rays", "n_sweeps", "n_steps"):
        assert a[k] == b[k], (what, k)
    np.testing.assert_array_equal(np_(a["band_flux"]), np_(b["band_flux"]))


def same_batched(a, b, what):
    """As `same`, but band fluxes of batched renders are FP64 atomic sums
    (equal up to summation order)."""
    for k in KEYS:
        x, y = np_(a[k]), np_(b[k])
        assert x.shape == y.shape and (x == y).all(), (what, k)
    for k in ("n_out", "n_leaves", "n_rays", "n_sweeps", "n_steps"):
        assert a[k] == b[k], (what, k)
    np.testing.assert_allclose(np_(a["band_flux"]), np_(b["band_flux"]), rtol=1e-12)


def test_training_reduced_the_loss(setup):
    s, g, net, hist = setup
    assert hist[-1] < 0.7 * hist[0]


@pytest.mark.parametrize("q", [0.05, 0.5, 0.8, 1.0])
def test_learned_image_equals_plain(setup, q):
    s, g, net, _ = setup
    for v in scenes.random_views(77, 3) + [scenes.axis_view("-z")]:
        plain = g.render_adaptive(v, N0, LM, XC, include_interior=True)
        got, st = g.render_learned(v, N0, LM, XC, net, quantile=q, include_interior=True)
        same(got, plain, f"q {q}")
        assert st["used_rays"] + st["wasted_rays"] == st["proposed_rays"]
        assert plain["n_rays"] == N0 * N0 + st["used_rays"] + st["fallback_rays"]


def test_untrained_network_still_exact(setup):
    s, g, _, _ = setup
    zero = air.MLP(np.zeros(air.MLP_NPARAMS, np.float32))
    v = scenes.random_views(78, 1)[0]
    plain = g.render_adaptive(v, N0, LM, XC)
    got, st = g.render_learned(v, N0, LM, XC, zero, quantile=0.8)
    same(got, plain, "zero network")
    zero.close()


def test_labels_are_the_oracle_tree_depths(setup):
    s, g, _, _ = setup
    o = oracle.Oracle(s)
    v = scenes.axis_view("+z")
    x, y = g.learn_samples(v, N0, LM, XC)
    t = o.air(v, N0, LM, XC)
    # sample 4 b + q: the deepest level below level-1 pixel q of base pixel b
    depth = np.zeros(4 * N0 * N0, int)
    for L, i, j in zip(t["level"], t["i"], t["j"]):
        if L == 0:
            continue
        b = (j >> L) * N0 + (i >> L)
        q = ((i >> (L - 1)) & 1) + 2 * ((j >> (L - 1)) & 1)
        depth[4 * b + q] = max(depth[4 * b + q], L)
    assert (np_(y) == depth).all()
    f = np_(x).view(np.uint16).astype(np.uint32) << 16
    feats = f.view(np.float32).reshape(4 * N0 * N0, 16)
    assert np.isfinite(feats).all() and (feats[:, 15] == 1.0).all()
    assert ((feats[:, 0] >= 0) & (feats[:, 0] <= 1)).all()


def test_trained_network_saves_waves(setup):
    s, g, net, _ = setup
    zero = air.MLP(np.zeros(air.MLP_NPARAMS, np.float32))
    waves_t, waves_plain, waste_t, waste_z = [], [], [], []
    for v in scenes.random_views(99, 6):
        plain = g.render_adaptive(v, N0, LM, XC)
        _, st = g.render_learned(v, N0, LM, XC, net, quantile=0.8)
        _, sz = g.render_learned(v, N0, LM, XC, zero, quantile=0.8)
        waves_t.append(st["waves"])
        waves_plain.append(1 + plain["n_sweeps"])
        waste_t.append(st["wasted_rays"] / max(plain["n_rays"], 1))
        waste_z.append(sz["wasted_rays"] / max(plain["n_rays"], 1))
    assert np.mean(waves_t) < np.mean(waves_plain)
    assert np.mean(waste_t) < np.mean(waste_z)
    zero.close()


@pytest.mark.parametrize("q,bpt", [(0.8, 0), (0.3, 1), (1.0, 2)])
def test_batched_learned_equals_plain_batched(setup, q, bpt):
    """air_render_batch_learned: every view's image is bitwise the plain
    batched render's (itself equal to the single-view render), whatever the
    proposal quantile and band split; the proposal traces most of the image
    in its wave."""
    s, g, net, hist = setup
    vs = [scenes.axis_view("+z")] + scenes.random_views(77, 4)
    plain = g.render_batch(vs, N0, LM, XC, include_interior=True, bands_per_thread=bpt)
    lrn, st = g.render_batch_learned(vs, N0, LM, XC, net, quantile=q, include_interior=True,
                                     bands_per_thread=bpt)
    for k, (a, b) in enumerate(zip(lrn, plain)):
        same_batched(a, b, f"view {k} q {q} bpt {bpt}")
    traced = sum(r["n_rays"] - N0 * N0 for r in plain)
    assert st["used_rays"] + st["fallback_rays"] == traced
    assert st["used_rays"] + st["wasted_rays"] == st["proposed_rays"]
    if q <= 0.8:
        assert st["used_rays"] > 0.5 * traced, st


def test_batched_learned_large_view_count(setup):
    """Twenty views in one batched learned render: same images as plain batched."""
    s, g, net, hist = setup
    vs = scenes.random_views(91, 20)
    plain = g.render_batch(vs, N0, LM, XC)
    lrn, st = g.render_batch_learned(vs, N0, LM, XC, net)
    for k, (a, b) in enumerate(zip(lrn, plain)):
        same_batched(a, b, f"view {k}")
