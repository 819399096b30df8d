"""FP64 reference of the refinement-depth MLP -- test infrastructure.

Only tests/ and the benchmark's baseline leg use this module; the CUDA library
never imports it. Plain numpy: a 3-layer perceptron 16 -> 64 -> 64 -> 5 with
ReLU, softmax cross-entropy averaged over the samples, its gradient by the
chain rule written out layer by layer, and the Adam update (Kingma & Ba 2015,
Algorithm 1). Parameters are one flat vector in the order
W1[16,64], b1[64], W2[64,64], b2[64], W3[64,5], b3[5] (row-major, input index
first).

`bf16=True` reproduces the GPU kernels' operand precision: the inputs, the
weights of every layer and the hidden activations after ReLU are rounded to
bfloat16 (round to nearest, ties to even, on the float32 bit pattern) before
each product, and so are the back-propagated deltas where they multiply a
weight matrix (d3 before d3 W3^T, d2 before d2 W2^T); the weight gradients use
the unrounded deltas. Sums are FP64 here and FP32 on the GPU.
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 16, 64, 5
SHAPES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (NH, NOUT)), ("b3", (NOUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[n], dtype=np.float64).ravel() for n, _ in SHAPES])


def bf16_round(x):
    """float -> nearest bfloat16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, bf16=False):
    p = unpack(theta)
    q = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = q(X)
    z1 = x @ q(p["W1"]) + p["b1"]
    h1 = q(np.maximum(z1, 0.0))
    z2 = h1 @ q(p["W2"]) + p["b2"]
    h2 = q(np.maximum(z2, 0.0))
    logits = h2 @ q(p["W3"]) + p["b3"]
    return logits, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, p=p, q=q)


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss_grad(theta, X, y, bf16=False):
    """Mean softmax cross-entropy and its gradient with respect to theta."""
    logits, c = forward(theta, X, bf16)
    n = len(y)
    P = softmax(logits)
    loss = -np.mean(np.log(P[np.arange(n), y]))
    d3 = P.copy()
    d3[np.arange(n), y] -= 1.0
    d3 /= n
    q, p = c["q"], c["p"]
    g = {}
    g["W3"] = c["h2"].T @ d3
    g["b3"] = d3.sum(axis=0)
    d2 = (q(d3) @ q(p["W3"]).T) * (c["z2"] > 0)
    g["W2"] = c["h1"].T @ d2
    g["b2"] = d2.sum(axis=0)
    d1 = (q(d2) @ q(p["W2"]).T) * (c["z1"] > 0)
    g["W1"] = c["x"].T @ d1
    g["b1"] = d1.sum(axis=0)
    return loss, pack(g)


def adam(theta, m, v, g, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new theta, m, v."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
