"""Sensitivity of truncated one-site TDVP-PS to rounding-like perturbations of its matvecs (CPU,
oracle only).

A property of the method, not a pin of its arithmetic.  Every element of every H_eff and H0
matvec is multiplied by (1 + eps z), z complex Gaussian: a relative perturbation that keeps exact
zeros exact, as rounding does.  From the product start at a truncated bond dimension:
- at the gauge shift's rank threshold 1e-6 the population drift over 50 steps is proportional to
  eps (no rank decision flips: the residuals near the threshold are far above the perturbation);
- with the threshold at 1e-13, near the perturbed residuals, the same perturbation drifts more
  than ten times as far (decisions flip).
"""
import numpy as np

import workloads as wl
import oracle.tdvp as T
from oracle import TDVPState, tdvp_ps_step, populations
from oracle.mps import heff_apply as HEFF, h0_apply as H0


def _drift(monkeypatch, eps, rtol, steps=50, D=16):
    rng = np.random.default_rng(0)

    def noisy(f):
        def g(*a):
            y = f(*a)
            return y * (1 + eps * (rng.normal(size=y.shape) + 1j * rng.normal(size=y.shape)))
        return g
    p = wl.tiny_chain()
    runs = []
    for e in (0.0, eps):
        monkeypatch.setattr(T, "heff_apply", noisy(HEFF) if e else HEFF)
        monkeypatch.setattr(T, "h0_apply", noisy(H0) if e else H0)
        st = TDVPState.start(p, D=D)
        P = []
        for _ in range(steps):
            tdvp_ps_step(st, 10.0, tol=1e-10, rank_rtol=rtol)
            P.append(populations(st, p))
        runs.append(np.array(P))
    return float(np.abs(runs[1] - runs[0]).max())


def test_drift_is_proportional_to_the_perturbation_away_from_the_rank_threshold(monkeypatch):
    large = _drift(monkeypatch, 2e-7, 1e-6)
    small = _drift(monkeypatch, 2e-11, 1e-6)
    # measured: 3.3e-7 and 3.3e-11
    assert 1e3 <= large / small <= 1e5, (large, small)
    near = _drift(monkeypatch, 2e-7, 1e-13)
    # measured: 9.9e-6
    assert near > 10 * large, (near, large)
