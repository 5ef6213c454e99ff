"""float64 reference of the variant-selector MLP -- TEST INFRASTRUCTURE ONLY.

Network: x (12 features) -> Linear(12, 64) -> ReLU -> Linear(64, 64) -> ReLU ->
Linear(64, 11); loss = (1 / batch) * sum over samples and outputs of
mask * (y - t)^2 (outputs without a target have mask 0). Weights are row-major
[out][in]. This is the plain
textbook definition of a two-hidden-layer perceptron with a masked squared
error; the CUDA kernels are checked against it and it is checked against
central finite differences.
"""
from __future__ import annotations

import numpy as np

D_IN, D_H, D_OUT = 12, 64, 11
SHAPES = [("w1", (D_H, D_IN)), ("b1", (D_H,)), ("w2", (D_H, D_H)), ("b2", (D_H,)),
          ("w3", (D_OUT, D_H)), ("b3", (D_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[n], dtype=np.float64).ravel() for n, _ in SHAPES])


def forward(theta: np.ndarray, x: np.ndarray):
    p = unpack(np.asarray(theta, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["w1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["w2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"].T + p["b3"]
    return y, (x, z1, h1, z2, h2)


def loss(theta, x, t, mask) -> float:
    y, _ = forward(theta, x)
    d = (y - t) * mask
    return float(np.sum(d * d) / max(1, x.shape[0]))


def grad(theta, x, t, mask):
    """Analytic gradient of ``loss`` by the chain rule."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    y, (x, z1, h1, z2, h2) = forward(theta, x)
    b = max(1, x.shape[0])
    dy = 2.0 * (y - t) * mask / b
    g = {"w3": dy.T @ h2, "b3": dy.sum(0)}
    dh2 = dy @ p["w3"]
    dz2 = dh2 * (z2 > 0)
    g["w2"], g["b2"] = dz2.T @ h1, dz2.sum(0)
    dh1 = dz2 @ p["w2"]
    dz1 = dh1 * (z1 > 0)
    g["w1"], g["b1"] = dz1.T @ x, dz1.sum(0)
    return loss(theta, x, t, mask), pack(g)


def sgd_step(theta, gradient, lr):
    return theta - lr * gradient


def adam_step(theta, gradient, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; step counts from 1."""
    m = beta1 * m + (1 - beta1) * gradient
    v = beta2 * v + (1 - beta2) * gradient * gradient
    mh = m / (1 - beta1**step)
    vh = v / (1 - beta2**step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
