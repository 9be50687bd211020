"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches them.

The detector is the exactness of TDVP-PS at maximal bond dimension on the tiny
chain, plus the closed-form Rabi oscillation for unit and sign slips.
"""
import numpy as np
import pytest

import workloads as wl
import oracle.tdvp as T
from oracle import TDVPState, tdvp_ps_step, populations
from oracle.dense import hamiltonian_kron, product_state, propagate_exact, populations_dense


def _exact_error(steps=3):
    p = wl.tiny_chain()
    st = TDVPState.start(p, D=32)
    exact = propagate_exact(hamiltonian_kron(p), product_state(p), 10.0 * np.arange(1, steps + 1))
    worst = 0.0
    for s in range(steps):
        tdvp_ps_step(st, 10.0)
        worst = max(worst, np.abs(populations(st, p) - populations_dense(exact[s], p)).max())
    return worst


def test_detector_is_quiet_without_a_mistake():
    assert _exact_error() < 1e-12


def test_backward_sign_flip_is_caught(monkeypatch):
    orig = T.lanczos_expm

    def flipped(matvec, v, z, *a, **k):
        if v.ndim == 2:                       # the bond (zero-site) evolution
            z = -z
        return orig(matvec, v, z, *a, **k)
    monkeypatch.setattr(T, "lanczos_expm", flipped)
    assert _exact_error() > 1e-4


def test_bra_ket_swap_in_left_environment_is_caught(monkeypatch):
    orig = T.heff_apply
    monkeypatch.setattr(T, "heff_apply", lambda L, W, R, A: orig(L.transpose(2, 1, 0), W, R, A))
    assert _exact_error() > 1e-4


def test_dropped_mpo_term_is_caught(monkeypatch):
    orig = T.build_mpo

    def no_coupling(p):
        W = orig(p)
        W[1] = W[1].copy()
        W[1][4, 1] = 0.0                      # drop the g w (b^+ + b) n block of the first mode
        return W
    monkeypatch.setattr(T, "build_mpo", no_coupling)
    assert _exact_error() > 1e-4


def test_half_step_at_turning_site_is_caught(monkeypatch):
    orig = T.lanczos_expm
    calls = {"n": 0}

    def halve_last(matvec, v, z, *a, **k):
        calls["n"] += 1
        if calls["n"] % 21 == 11:             # 10 calls per half sweep on 6 sites: the 11th is site N
            assert v.ndim == 3
            z = z / 2
        return orig(matvec, v, z, *a, **k)
    monkeypatch.setattr(T, "lanczos_expm", halve_last)
    assert _exact_error() > 1e-6


def test_wrong_time_unit_is_caught(monkeypatch):
    monkeypatch.setattr(T, "PHASE_PER_CM_FS", T.PHASE_PER_CM_FS * 1.01)
    p = wl.two_level_rabi()
    st = TDVPState.start(p, D=2)
    for _ in range(10):
        tdvp_ps_step(st, 10.0)
    Om = np.sqrt((p.E[0] - p.E[1]) ** 2 + 4 * p.J[0, 1] ** 2)
    t = 100.0 * 2 * np.pi * 2.99792458e-5
    P1 = 1 - 4 * p.J[0, 1] ** 2 / Om ** 2 * np.sin(Om * t / 2) ** 2
    assert abs(populations(st, p)[0] - P1) > 1e-6



# ---------------------------------------------------------------- observables: the dense-state pin

def _obs_deviation(**mutated):
    from test_oracle_pins import _dense_observable_deviation
    return _dense_observable_deviation(wl.tiny_chain(), 8, 21, **mutated)


def _energy_unnormalised(st):
    """energy() with the division by <Psi|Psi> left out."""
    E = np.ones((1, 1, 1), dtype=complex)
    for A, W in zip(st.mps, st.W):
        E = T.env_left(E, A, W)
    return float(E[0, 0, 0].real)


def _mpo_without_first_coupling(p):
    W = T.build_mpo(p)
    W[1] = W[1].copy()
    W[1][4, 1] = 0.0                          # the g w (b^+ + b) n block of the first mode
    return W


def test_observable_pin_is_quiet_without_a_mistake():
    assert _obs_deviation() < 1e-12


def test_energy_without_normalisation_is_caught():
    assert _obs_deviation(energy_fn=_energy_unnormalised) > 1e-3


def test_energy_with_dropped_mpo_term_is_caught():
    assert _obs_deviation(mpo_fn=_mpo_without_first_coupling) > 1e-6


def test_norm_without_square_root_is_caught():
    assert _obs_deviation(norm_fn=lambda st: float(abs(T._expect_local(st.mps, {})))) > 1e-3


def test_norm_that_is_always_one_is_caught():
    assert _obs_deviation(norm_fn=lambda st: 1.0) > 1e-3


def test_populations_without_normalisation_is_caught():
    def unnormalised(st, p):
        return T.populations(st, p) * T._expect_local(st.mps, {}).real
    assert _obs_deviation(pops_fn=unnormalised) > 1e-3
