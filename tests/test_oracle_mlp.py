"""Pins of the reference MLP: each head's backward pass equals central finite differences of its
loss, the acceptance gradient is confined to the acceptance head, and the label rule is the
closed form [k <= floor(y)] on a network whose output is a known constant."""
import numpy as np
import pytest

from oracle import mlp


@pytest.mark.parametrize("head", [0, 1])
def test_reference_mlp_gradient_equals_finite_differences(head):
    rng = np.random.default_rng(3 + head)
    w = mlp.init(1)
    X = rng.normal(size=(17, mlp.NIN))
    t = rng.uniform(2, 20, size=17) if head == 0 else rng.integers(1, 12, size=17).astype(float)
    L, g = mlp.loss_and_grad(w, X, t, head)
    idx = rng.choice(mlp.NPARAM, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, mlp.NPARAM - 2, mlp.NPARAM - 66, 0, 8 * 64 + 3]])
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        # the acceptance labels are a step function of y: hold them at w's values
        fd = (mlp.loss_and_grad(wp, X, t, head)[0] - mlp.loss_and_grad(wm, X, t, head)[0]) / (2 * h)
        if head == 1 and i < mlp.NPARAM - 65:
            assert g[i] == 0.0                   # the trunk and head 1 are frozen in this stage
            continue
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert mlp.NPARAM == 4866


def test_acceptance_labels_follow_the_used_dimension():
    """With the trunk output fixed (zero hidden weights) y = b3, so kp = floor(b3) clamped; the
    labels are [k <= kp] and the loss with a = b4 is the logistic loss of those labels."""
    p = mlp.unpack(mlp.init(2))
    for k in ("W1", "W2", "W3", "W4"):
        p[k] = np.zeros_like(p[k])
    p["b3"] = np.array([6.7])
    p["b4"] = np.array([0.3])
    w = mlp.pack(p)
    X = np.random.default_rng(4).normal(size=(8, mlp.NIN))
    t = np.array([1, 5, 6, 7, 8, 6, 2, 9], float)
    assert np.all(mlp.used_dimension(w, X) == 6)
    lab = (t <= 6).astype(float)
    L, _ = mlp.loss_and_grad(w, X, t, head=1)
    assert abs(L - np.mean(np.log1p(np.exp(0.3)) - lab * 0.3)) < 1e-12
