"""FP64 reference of the reaction surrogate: a 8 -> 64 -> 64 -> 8 perceptron
with ReLU hidden layers, its mean-squared-error loss, analytic gradients
(backpropagation) and the Adam update.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain NumPy in float64,
written from the definitions: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3,
L = (1/(B*O)) sum_i |y_i - t_i|^2, Adam as in Kingma & Ba (2015).  The paper
has no surrogate; this is the learned part of the reaction substep that
replaces the exact cell-model update where allowed.

Shapes: W1 [64, 8], b1 [64], W2 [64, 64], b2 [64], W3 [8, 64], b3 [8];
x [B, 8], t [B, 8].
"""
from __future__ import annotations

import numpy as np

SIZES = (8, 64, 64, 8)


def init_params(seed, sizes=SIZES):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for i, (a, b) in enumerate(zip(sizes[:-1], sizes[1:]), start=1):
        r = 1.0 / np.sqrt(a)
        p["W%d" % i] = rng.uniform(-r, r, size=(b, a))
        p["b%d" % i] = np.zeros(b)
    return p


def forward(p, x):
    """Returns the output and the hidden activations."""
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(x @ p["W1"].T + p["b1"], 0.0)
    h2 = np.maximum(h1 @ p["W2"].T + p["b2"], 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, h1, h2)


def loss(p, x, t):
    y, _ = forward(p, x)
    d = y - np.asarray(t, dtype=np.float64)
    return float(np.mean(d * d))


def grads(p, x, t):
    """Analytic gradient of `loss` with respect to every parameter."""
    y, (x, h1, h2) = forward(p, x)
    B, O = y.shape
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / (B * O)
    g = {"W3": dy.T @ h2, "b3": dy.sum(axis=0)}
    dh2 = (dy @ p["W3"]) * (h2 > 0)  # relu'(z) = 1 for z > 0, else 0
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"]) * (h1 > 0)
    g["W1"] = dh1.T @ x
    g["b1"] = dh1.sum(axis=0)
    return g


def pack(p):
    """Parameters as one float vector in the order W1, b1, W2, b2, W3, b3
    (row-major matrices), the layout of the library's MLP entry points."""
    return np.concatenate([p[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unpack(vec, sizes=SIZES):
    vec = np.asarray(vec, dtype=np.float64)
    p, o = {}, 0
    for i, (a, b) in enumerate(zip(sizes[:-1], sizes[1:]), start=1):
        p["W%d" % i] = vec[o:o + a * b].reshape(b, a); o += a * b
        p["b%d" % i] = vec[o:o + b].copy(); o += b
    assert o == vec.size
    return p


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; step counts from 1."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mh = m[k] / (1 - beta1 ** step)
        vh = v[k] / (1 - beta2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
