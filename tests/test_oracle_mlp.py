"""Pins for the FP64 MLP reference (oracle/mlp.py): finite differences of its
own loss pin the hand-written backward pass; closed forms pin the loss, the
softmax gradient and Adam's first step; bfloat16 rounding is checked on values
whose rounding is fixed by the format (8 exponent bits, 7 stored mantissa bits,
round to nearest, ties to even)."""
import math

import numpy as np
import pytest

from oracle import mlp
import scenes


def _data(seed, n=40):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, mlp.NIN))
    y = rng.integers(0, mlp.NOUT, size=n)
    return X, y


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences(seed):
    X, y = _data(seed)
    th = scenes.mlp_init(seed, scale=0.7)
    th[mlp.NPARAMS - 5:] = np.random.default_rng(seed).normal(size=5) * 0.1  # nonzero b3
    loss, g = mlp.loss_grad(th, X, y)
    rng = np.random.default_rng(seed + 10)
    idx = rng.choice(mlp.NPARAMS, size=120, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.NPARAMS)
        e[k] = h
        fd = (mlp.loss_grad(th + e, X, y)[0] - mlp.loss_grad(th - e, X, y)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-8), k


def test_zero_parameters_closed_form():
    X, y = _data(3)
    th = np.zeros(mlp.NPARAMS)
    loss, g = mlp.loss_grad(th, X, y)
    assert loss == pytest.approx(math.log(5.0), rel=1e-15)
    gb3 = g[mlp.NPARAMS - 5:]
    expect = np.full(5, 0.2) - np.bincount(y, minlength=5) / len(y)
    np.testing.assert_allclose(gb3, expect, rtol=1e-14, atol=1e-16)
    assert np.all(g[:mlp.NPARAMS - 5] == 0.0)


def test_adam_first_step_is_sign_step():
    th = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    new, m, v = mlp.adam(th, np.zeros(3), np.zeros(3), g, lr=0.01, t=1)
    np.testing.assert_allclose(new, th - 0.01 * np.sign(g), rtol=0, atol=1e-7)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_bf16_rounding_values():
    vals = {1.0: 1.0, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6, 1 + 2 ** -7: 1 + 2 ** -7,
            3.14159: 3.140625, -2.5: -2.5, 65535.0: 65536.0, 1e-3: 0.00099945068359375}
    for x, r in vals.items():
        assert mlp.bf16_round(np.array([x]))[0] == r, x


def test_bf16_mode_is_close_to_fp64_and_training_learns():
    X, y = _data(5, n=200)
    th = scenes.mlp_init(5, scale=0.5)
    l64, g64 = mlp.loss_grad(th, X, y)
    l16, g16 = mlp.loss_grad(th, X, y, bf16=True)
    assert abs(l16 - l64) < 2e-2 * l64
    assert np.linalg.norm(g16 - g64) < 5e-2 * np.linalg.norm(g64)
    # labels a function of the inputs: training must reduce the loss
    yt = (X[:, 0] > 0).astype(int) + 2 * (X[:, 1] > 0).astype(int)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    first = mlp.loss_grad(th, X, yt)[0]
    for t in range(1, 201):
        _, g = mlp.loss_grad(th, X, yt)
        th, m, v = mlp.adam(th, m, v, g, 1e-2, t)
    assert mlp.loss_grad(th, X, yt)[0] < 0.3 * first
