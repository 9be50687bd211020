"""Pin of the reference MLP: its backward pass equals central finite differences of its loss."""
import numpy as np

from oracle import mlp


def test_reference_mlp_gradient_equals_finite_differences():
    rng = np.random.default_rng(3)
    w = mlp.init(1)
    X = rng.normal(size=(17, mlp.NIN))
    t = rng.uniform(2, 20, size=17)
    L, g = mlp.loss_and_grad(w, X, t)
    idx = rng.choice(mlp.NPARAM, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 0, 8 * 64 + 3]])
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_and_grad(wp, X, t)[0] - mlp.loss_and_grad(wm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert mlp.NPARAM == 4801
