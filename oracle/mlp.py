"""Plain FP64 reference of the coefficient surrogate network (TEST INFRASTRUCTURE ONLY).

The surrogate is a 3 -> 64 -> 64 -> 3 multilayer perceptron with SiLU activations:
    z1 = W1 x + b1, h1 = silu(z1), z2 = W2 h1 + b2, h2 = silu(z2), y = W3 h2 + b3,
silu(z) = z / (1 + e^{-z}).  The loss is the masked mean squared error
    L = sum_{n,k} m_nk (y_nk - t_nk)^2 / sum_{n,k} m_nk.
This module writes the forward pass and the gradients of L by the chain rule, in numpy
float64, one line per step of the definition; the tests pin the gradients against central
finite differences and then use them to check the CUDA training kernels.
Weights are a dict with W1 [64,3], b1 [64], W2 [64,64], b2 [64], W3 [3,64], b3 [3].
"""
from __future__ import annotations

import numpy as np

SHAPES = {"W1": (64, 3), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (3, 64), "b3": (3,)}


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init(seed=0):
    """Deterministic test weights (scaled normal)."""
    rng = np.random.default_rng(seed)
    w = {}
    for k, s in SHAPES.items():
        fan_in = s[1] if len(s) == 2 else 1
        w[k] = rng.standard_normal(s) / np.sqrt(fan_in) if len(s) == 2 else 0.1 * rng.standard_normal(s)
    return w


def forward(w, x):
    z1 = x @ w["W1"].T + w["b1"]
    h1 = silu(z1)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = silu(z2)
    y = h2 @ w["W3"].T + w["b3"]
    return y, (x, z1, h1, z2, h2)


def loss(w, x, t, m):
    y, _ = forward(w, x)
    return float(np.sum(m * (y - t) ** 2) / np.sum(m))


def grad(w, x, t, m):
    """Gradients of the masked mean squared error with respect to every weight and bias."""
    y, (x, z1, h1, z2, h2) = forward(w, x)
    dy = 2.0 * m * (y - t) / np.sum(m)          # dL/dy
    g = {}
    g["W3"] = dy.T @ h2                          # dL/dW3 = sum_n dy_n h2_n^T
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ w["W3"]                           # dL/dh2
    dz2 = dh2 * dsilu(z2)                        # through silu
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ w["W2"]
    dz1 = dh1 * dsilu(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return g
