"""Reference two-layer MLP of the Krylov controller: 8 -> 64 -> 64 (ReLU) with two heads.

TEST INFRASTRUCTURE (oracle); see the package docstring.  Plain numpy forward and backward
written from the chain rule, in float64, used to check the gradients of the GPU training kernels.
Head 1 is the Krylov dimension y (linear, mean-squared error); head 2 the logit a of accepting
kp = floor(y) clamped to [1, 126], trained on the label [k <= kp] by the logistic loss with the
trunk frozen (its gradient covers head 2 only).  The label is an integer decision taken from a
floating-point y, so it is taken in the precision of the GPU network (float32).
Parameter vector layout (4866 values): W1[8][64], b1[64], W2[64][64], b2[64], W3[64], b3, W4[64], b4.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 8, 64
SIZES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)), ("b3", (1,)),
         ("W4", (NH,)), ("b4", (1,))]
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
    """Both heads: y (Krylov dimension) and a (acceptance logit), with the hidden activations."""
    p = unpack(w)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"][0]
    a = h2 @ p["W4"] + p["b4"][0]
    return y, a, (X, z1, h1, z2, h2)


def used_dimension(w, X):
    """kp = floor(y) clamped to [1, 126], with y evaluated in float32 (the GPU network's precision)."""
    p = {k: v.astype(np.float32) for k, v in unpack(w).items()}
    X = np.asarray(X, dtype=np.float32)
    h1 = np.maximum(X @ p["W1"] + p["b1"], np.float32(0))
    h2 = np.maximum(h1 @ p["W2"] + p["b2"], np.float32(0))
    y = h2 @ p["W3"] + p["b3"][0]
    return np.clip(np.floor(y), 1, 126)


def loss_and_grad(w, X, t, head=0):
    """head 0: L = mean (y - t)^2 and dL/dw (trunk and head 1); head 1: L = mean logistic loss of
    sigma(a) against [t <= kp] and dL/dw (head 2 only, zero elsewhere)."""
    p = unpack(w)
    y, a, (X, z1, h1, z2, h2) = forward(w, X)
    B = X.shape[0]
    g = {name: np.zeros(shape) for name, shape in SIZES}
    if head == 1:
        lab = (np.asarray(t) <= used_dimension(w, X)).astype(np.float64)
        L = float(np.mean(np.logaddexp(0.0, a) - lab * a))
        da = (1.0 / (1.0 + np.exp(-a)) - lab) / B
        g["W4"] = h2.T @ da
        g["b4"] = np.array([da.sum()])
        return L, pack(g)
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / B
    g["W3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
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
         "W3": rng.normal(0, np.sqrt(1.0 / NH), NH), "b3": np.array([4.0]),
         "W4": rng.normal(0, np.sqrt(1.0 / NH), NH), "b4": np.array([0.5])}
    return pack(p)
