"""GPU refinement-depth network (tensor-core mma.sync BF16 kernels) against the
FP64 reference oracle/mlp.py. With the reference in its BF16-operand mode the
differences left are FP32 versus FP64 accumulation and, in the weight
gradients, the back-propagated errors carried as two BF16 parts (about 16
significant bits, <= 2^-16 relative per term), so logits agree to ~1e-5 and
gradients well inside 2e-3 of their scale; against the plain FP64 network
the BF16 bound (~3e-2 of the gradient norm) applies."""
import numpy as np
import pytest

import paper_1010_5534_gb300 as air
from oracle import mlp
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _bits(Xq):
    return torch.from_numpy(np.ascontiguousarray(Xq.astype(np.float32)).view(np.uint32) >> 16)\
        .to(torch.int32).to(torch.int16).cuda()


def _data(seed, n):
    rng = np.random.default_rng(seed)
    Xq = mlp.bf16_round(rng.normal(size=(n, mlp.NIN)))
    y = rng.integers(0, mlp.NOUT, size=n)
    return Xq, y


@pytest.fixture(scope="module", autouse=True)
def _b():
    air.build()


@pytest.mark.parametrize("n", [1, 37, 128, 1000])
def test_forward_matches_reference(n):
    th = scenes.mlp_init(3, scale=0.8)
    th[mlp.NPARAMS - 5:] = [0.1, -0.2, 0.3, 0.0, 0.05]
    th = th.astype(np.float32).astype(np.float64)
    Xq, _ = _data(n, n)
    net = air.MLP(th)
    lg = net.forward(_bits(Xq)).cpu().numpy().astype(np.float64)
    ref, _ = mlp.forward(th, Xq, bf16=True)
    np.testing.assert_allclose(lg, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    net.close()


@pytest.mark.parametrize("n", [128, 300, 2049])
def test_gradient_matches_reference(n):
    th = scenes.mlp_init(4, scale=0.8).astype(np.float32).astype(np.float64)
    Xq, y = _data(n + 1, n)
    net = air.MLP(th)
    loss, g = net.loss_grad(_bits(Xq), torch.from_numpy(y.astype(np.int32)).cuda())
    g = g.cpu().numpy().astype(np.float64)
    l16, g16 = mlp.loss_grad(th, Xq, y, bf16=True)
    assert loss == pytest.approx(l16, rel=1e-5)
    scale = np.abs(g16).max()
    np.testing.assert_allclose(g, g16, rtol=2e-3, atol=2e-4 * scale)
    l64, g64 = mlp.loss_grad(th, Xq, y, bf16=False)
    assert np.linalg.norm(g - g64) < 3e-2 * np.linalg.norm(g64)
    assert np.dot(g, g64) / (np.linalg.norm(g) * np.linalg.norm(g64)) > 0.999
    net.close()


def test_adam_steps_match_reference():
    th = scenes.mlp_init(5, scale=0.8).astype(np.float32).astype(np.float64)
    Xq, y = _data(9, 512)
    net = air.MLP(th)
    xd, yd = _bits(Xq), torch.from_numpy(y.astype(np.int32)).cuda()
    net.train(xd, yd, batch=512, epochs=3, lr=1e-2)
    got = net.params().astype(np.float64)
    ref, m, v = th.copy(), np.zeros_like(th), np.zeros_like(th)
    for t in range(1, 4):
        _, g = mlp.loss_grad(ref.astype(np.float32).astype(np.float64), Xq, y, bf16=True)
        ref, m, v = mlp.adam(ref, m, v, g, 1e-2, t)
    # Adam normalises the step, so parameters agree to ~lr x (relative gradient error)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-3)
    net.close()


def test_training_learns_a_separable_rule():
    rng = np.random.default_rng(11)
    n = 16384
    Xq = mlp.bf16_round(rng.normal(size=(n, mlp.NIN)))
    y = np.clip((Xq[:, 0] > 0).astype(int) + (Xq[:, 1] > 0.5).astype(int) + 2 * (Xq[:, 2] > 1.0), 0, 4)
    net = air.MLP(scenes.mlp_init(6, scale=1.0))
    hist = net.train(_bits(Xq), torch.from_numpy(y.astype(np.int32)).cuda(), batch=1024,
                     epochs=16, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]
    pred = net.forward(_bits(Xq)).cpu().numpy().argmax(axis=1)
    assert (pred == y).mean() > 0.9
    net.close()
