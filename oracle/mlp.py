"""Reference two-layer MLP (8 -> 64 -> 64 -> 1, ReLU, mean-squared error) for the Krylov controller.

TEST INFRASTRUCTURE (oracle); see the package docstring.  Plain numpy forward and backward
written from the chain rule, in float64, used to check the gradients of the GPU training kernels.
Parameter vector layout (4801 values): W1[8][64], b1[64], W2[64][64], b2[64], W3[64], b3.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 8, 64
SIZES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = w[o:o + n].reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(w, X):
    p = unpack(w)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(w, X, t):
    """L = mean (y - t)^2 and dL/dw by the chain rule."""
    p = unpack(w)
    y, (X, z1, h1, z2, h2) = forward(w, X)
    B = X.shape[0]
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / B
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["W3"]) * (z2 > 0)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"].T) * (z1 > 0)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def init(seed=0):
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, np.sqrt(2.0 / NIN), (NIN, NH)), "b1": np.zeros(NH),
         "W2": rng.normal(0, np.sqrt(2.0 / NH), (NH, NH)), "b2": np.zeros(NH),
         "W3": rng.normal(0, np.sqrt(1.0 / NH), NH), "b3": np.array([4.0])}
    return pack(p)
