"""Pins of the P&C-RK4 oracle (Sec. II.A.1; Eq. mpo-apply, mps+mps, SVD, RK4) against dense
linear algebra, closed forms and exact propagation; CPU only.

- MPO x MPS against the Kronecker-built H applied to the dense state (the dense H is built term
  by term, independently of the MPO);
- MPS + MPS against the dense linear combination;
- compression without truncation keeps the state and leaves right-canonical sites;
- truncation of a state whose Schmidt decomposition is known by construction keeps exactly the
  largest terms (criterion i) or those above zeta (criterion ii);
- one untruncated RK4 step equals the degree-4 Taylor polynomial of exp(-i h H) (classical RK4
  on a linear autonomous equation), and its global error falls as h^4;
- the warm-up from the product state equals ten such dense steps, and its compressed state is
  normalised up to the RK4 error.
"""
import math

import numpy as np
import pytest

import workloads as wl
from workloads import PHASE_PER_CM_FS
from oracle import build_mpo, mps_to_dense, product_mps
from oracle.dense import hamiltonian_kron, product_state, propagate_exact
from oracle.pc_rk4 import (mpo_apply, mps_add, compress, rk4_step, warmup, canonicalise_left,
                           svd_compress, ATOMIC_TIME_FS)


def _small_vibronic():
    """3 electronic sites with 1-2 modes each (left- and right-indexed MPO channels)."""
    E = np.array([12400.0, 12450.0, 12300.0])
    J = np.array([[0, -60.0, 25.0], [-60.0, 0, 40.0], [25.0, 40.0, 0]])
    om = [np.array([150.0]), np.array([220.0, 480.0]), np.array([330.0])]
    g = [np.array([0.4]), np.array([0.3, 0.2]), np.array([0.5])]
    lev = [np.array([3]), np.array([3, 2]), np.array([3])]
    return wl.FHParams(E=E, J=J, omega=om, g=g, n_levels=lev, el_order=[2, 0, 1],
                       energy_offset=12400.0)


MODELS = [wl.tiny_chain, _small_vibronic]


def _taylor4(H, psi, h):
    """sum_{n=0}^{4} (-i h H)^n / n! psi."""
    out = psi.copy()
    term = psi.copy()
    for n in range(1, 5):
        term = (-1j * h) * (H @ term) / n
        out = out + term
    return out


@pytest.mark.parametrize("maker", MODELS)
def test_mpo_apply_equals_dense_hamiltonian_action(maker):
    p = maker()
    W = build_mpo(p)
    H = hamiltonian_kron(p)
    for D, seed in ((1, 3), (3, 4), (6, 5)):
        t = wl.random_mps_tensors(p.phys_dims(), D, seed=seed)
        ref = H @ mps_to_dense(t)
        got = mps_to_dense(mpo_apply(W, t))
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        assert all(B.shape[0] == Wi.shape[0] * A.shape[0] and B.shape[2] == Wi.shape[1] * A.shape[2]
                   for B, Wi, A in zip(mpo_apply(W, t), W, t))


def test_mps_add_equals_dense_linear_combination():
    p = wl.tiny_chain()
    d = p.phys_dims()
    states = [wl.random_mps_tensors(d, D, seed=s) for D, s in ((2, 1), (4, 2), (1, 3), (3, 4), (5, 5))]
    coefs = [0.3, -2.0j, 1.5 + 0.5j, 1.0, -0.25]
    for k in (1, 2, 5):
        ref = sum(c * mps_to_dense(s) for c, s in zip(coefs[:k], states[:k]))
        got = mps_add(coefs[:k], states[:k])
        assert np.abs(mps_to_dense(got) - ref).max() <= 1e-13 * np.abs(ref).max()
        assert got[1].shape[0] == sum(s[1].shape[0] for s in states[:k])
    one_site = [np.arange(3, dtype=complex).reshape(1, 3, 1)]
    assert np.allclose(mps_add([2.0, 1j], [one_site, one_site])[0].ravel(), (2 + 1j) * np.arange(3))


@pytest.mark.parametrize("maker", MODELS)
def test_compression_without_truncation_keeps_the_state(maker):
    """M above every rank: the state is unchanged, sites 2..N are right-canonical, and every
    bond is at most min(prod d left, prod d right) (the exact Schmidt rank bound)."""
    p = maker()
    d = p.phys_dims()
    W = build_mpo(p)
    t = mpo_apply(W, wl.random_mps_tensors(d, 4, seed=7))   # bonds w * 4, far above the ranks
    c = compress(t, 10_000)
    assert np.abs(mps_to_dense(c) - mps_to_dense(t)).max() <= 1e-12 * np.abs(mps_to_dense(t)).max()
    for A in c[1:]:
        M = A.reshape(A.shape[0], -1)
        assert np.allclose(M @ M.conj().T, np.eye(A.shape[0]), atol=1e-12)
    for i in range(1, len(d)):
        assert c[i].shape[0] <= min(math.prod(d[:i]), math.prod(d[i:]))


def _schmidt_state(lam, d1=6, d2=7, seed=3):
    """Two-site MPS sum_s lam_s u_s (x) v_s with orthonormal u_s, v_s, written NON-canonically
    (site 1 = v_s^T, site 0 = u_s lam_s scaled by a random invertible matrix and its inverse),
    with its dense terms."""
    rng = np.random.default_rng(seed)
    r = len(lam)
    U, _ = np.linalg.qr(rng.normal(size=(d1, r)) + 1j * rng.normal(size=(d1, r)))
    V, _ = np.linalg.qr(rng.normal(size=(d2, r)) + 1j * rng.normal(size=(d2, r)))
    G = rng.normal(size=(r, r)) + 1j * rng.normal(size=(r, r)) + 3 * np.eye(r)
    A0 = ((U * lam) @ G).reshape(1, d1, r)
    A1 = (np.linalg.inv(G) @ V.T).reshape(r, d2, 1)
    terms = [lam[s] * np.kron(U[:, s], V[:, s]) for s in range(r)]
    return [A0, A1], terms


def test_truncation_keeps_the_largest_schmidt_terms():
    """Eq. SVD at the one bond of a two-site state with known Schmidt values: criterion (i)
    keeps the M largest terms exactly, criterion (ii) those above zeta ||Lambda||."""
    lam = np.array([0.8, 0.5, 0.3, 0.1, 0.05])
    mps, terms = _schmidt_state(lam)
    for M in (1, 2, 3, 5):
        got = mps_to_dense(compress(mps, M))
        ref = sum(terms[:M])
        assert np.abs(got - ref).max() <= 1e-12
        assert abs(np.linalg.norm(mps_to_dense(mps) - got) ** 2 - np.sum(lam[M:] ** 2)) <= 1e-12
    nrm = np.linalg.norm(lam)
    for zeta in (0.2, 0.09):
        keep = int(np.sum(lam > zeta * nrm))
        got = mps_to_dense(compress(mps, 100, zeta))
        assert np.abs(got - sum(terms[:keep])).max() <= 1e-12


def test_compression_leaves_a_zero_state_at_bond_one():
    p = wl.tiny_chain()
    z = [0.0 * A for A in wl.random_mps_tensors(p.phys_dims(), 3, seed=2)]
    c = compress(z, 8)
    assert all(A.shape[0] == 1 for A in c[1:]) and np.abs(mps_to_dense(c)).max() == 0.0


@pytest.mark.parametrize("maker", MODELS)
def test_untruncated_rk4_step_is_the_fourth_order_taylor_polynomial(maker):
    """Classical RK4 on the linear equation dPsi/dt = -i H Psi is exactly
    sum_{n<=4} (-i h H)^n / n! Psi (Eq. RK4 with k_1..k_4 expanded)."""
    p = maker()
    W = build_mpo(p)
    H = hamiltonian_kron(p)
    t = wl.random_mps_tensors(p.phys_dims(), 3, seed=12)
    psi = mps_to_dense(t)
    for dt in (0.5, 4.0):
        ref = _taylor4(H, psi, dt * PHASE_PER_CM_FS)
        got = mps_to_dense(rk4_step(W, t, dt, 10_000))
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_rk4_global_error_is_fourth_order():
    """Against exact propagation over 40 fs: halving the step divides the error by ~16."""
    p = wl.tiny_chain()
    W = build_mpo(p)
    H = hamiltonian_kron(p)
    psi0 = product_state(p)
    exact = propagate_exact(H, psi0, [40.0])[0]
    start = product_mps(p.phys_dims(), [1] * (len(p.phys_dims()) + 1), p.occupied())
    errs = []
    for n in (8, 16, 32):
        s = start
        for _ in range(n):
            s = rk4_step(W, s, 40.0 / n, 10_000)
        errs.append(np.linalg.norm(mps_to_dense(s) - exact))
    for a, b in zip(errs, errs[1:]):
        assert 12.0 <= a / b <= 20.0, errs


def test_warmup_equals_dense_rk4_and_stays_normalised():
    """The paper's warm-up on the tiny chain at a bond large enough to be exact: ten RK4 steps
    of 80 a.u. from the product state equal ten dense Taylor steps; compressed to M_S = 4 the
    state keeps bonds <= 4 and its norm stays 1 up to the RK4 error."""
    p = wl.tiny_chain()
    H = hamiltonian_kron(p)
    full = warmup(p, M_S=10_000, M_max=10_000)
    psi = product_state(p)
    for _ in range(10):
        psi = _taylor4(H, psi, 80.0 * ATOMIC_TIME_FS * PHASE_PER_CM_FS)
    assert np.abs(mps_to_dense(full) - psi).max() <= 1e-12
    # RK4 at h ||H|| = 1.66 on this chain: 5.6e-5 from the exact state after the ten steps
    exact = propagate_exact(H, product_state(p), [800.0 * ATOMIC_TIME_FS])[0]
    assert np.linalg.norm(psi - exact) <= 1e-3
    small = warmup(p, M_S=4, M_max=10_000)
    assert max(A.shape[2] for A in small) <= 4
    assert abs(np.linalg.norm(mps_to_dense(small)) - 1.0) <= 1e-5
    assert np.linalg.norm(mps_to_dense(small) - exact) <= 1e-3


# ---------------------------------------------------------------- planted mistakes (CPU)

import oracle.pc_rk4 as P  # noqa: E402


def _taylor_gap():
    p = wl.tiny_chain()
    t = wl.random_mps_tensors(p.phys_dims(), 3, seed=12)
    ref = _taylor4(hamiltonian_kron(p), mps_to_dense(t), 4.0 * PHASE_PER_CM_FS)
    got = mps_to_dense(P.rk4_step(build_mpo(p), t, 4.0, 10_000))
    return np.abs(got - ref).max() / np.abs(ref).max()


def _truncation_gap():
    lam = np.array([0.8, 0.5, 0.3, 0.1, 0.05])
    mps, terms = _schmidt_state(lam)
    return max(np.abs(mps_to_dense(P.compress(mps, M)) - sum(terms[:M])).max() for M in (1, 2, 3))


def _mpo_gap():
    p = _small_vibronic()
    t = wl.random_mps_tensors(p.phys_dims(), 3, seed=4)
    ref = hamiltonian_kron(p) @ mps_to_dense(t)
    return np.abs(mps_to_dense(P.mpo_apply(build_mpo(p), t)) - ref).max() / np.abs(ref).max()


def test_pins_are_quiet_without_a_mistake():
    assert _taylor_gap() < 1e-12 and _truncation_gap() < 1e-12 and _mpo_gap() < 1e-13


def test_swapped_rk4_weights_are_caught(monkeypatch):
    orig = P.mps_add

    def swapped(coefs, states):
        if len(coefs) == 5:
            coefs = [coefs[0], coefs[2], coefs[1], coefs[4], coefs[3]]
        return orig(coefs, states)
    monkeypatch.setattr(P, "mps_add", swapped)
    assert _taylor_gap() > 1e-6


def test_full_step_for_the_last_stage_is_caught(monkeypatch):
    orig = P.mps_add
    seen = []

    def half(coefs, states):
        if len(coefs) == 2:
            seen.append(coefs[1])
            if len(seen) == 3:                  # the Psi + h k3 stage taken with h / 2
                coefs = [coefs[0], coefs[1] / 2]
        return orig(coefs, states)
    monkeypatch.setattr(P, "mps_add", half)
    assert _taylor_gap() > 1e-6


def test_coefficient_on_every_site_is_caught(monkeypatch):
    orig = P.mps_add

    def everywhere(coefs, states):
        scaled = [[c * A for A in s] for c, s in zip(coefs, states)]
        return orig([1.0] * len(coefs), scaled)
    monkeypatch.setattr(P, "mps_add", everywhere)
    assert _taylor_gap() > 1e-6


class _NumpyWithSvd:
    """numpy as seen by the oracle module, with its SVD replaced."""

    def __init__(self, svd):
        self.linalg = type("linalg", (), {"svd": staticmethod(svd), "qr": staticmethod(np.linalg.qr),
                                          "norm": staticmethod(np.linalg.norm)})

    def __getattr__(self, name):
        return getattr(np, name)


def test_absorbing_u_without_the_singular_values_is_caught(monkeypatch):
    def flat(a, full_matrices=True):
        U, S, Vh = np.linalg.svd(a, full_matrices=full_matrices)
        return U, np.where(S > 0, S[0], 0.0), Vh
    monkeypatch.setattr(P, "np", _NumpyWithSvd(flat))
    assert _truncation_gap() > 1e-3


def test_keeping_the_smallest_singular_values_is_caught(monkeypatch):
    def reversed_order(a, full_matrices=True):
        U, S, Vh = np.linalg.svd(a, full_matrices=full_matrices)
        return U[:, ::-1], S[::-1], Vh[::-1]
    monkeypatch.setattr(P, "np", _NumpyWithSvd(reversed_order))
    assert _truncation_gap() > 1e-3


def test_compressing_without_canonicalisation_is_caught(monkeypatch):
    monkeypatch.setattr(P, "canonicalise_left", lambda mps: [np.array(A, complex) for A in mps])
    assert _truncation_gap() > 1e-3


def test_inconsistent_bond_order_in_mpo_apply_is_caught(monkeypatch):
    def mixed(W, mps):
        out = []
        for i, (Wi, A) in enumerate(zip(W, mps)):
            wl_, wr, d, _ = Wi.shape
            spec = "wvts,asb->watvb" if i % 2 == 0 else "wvts,asb->awtbv"
            out.append(np.einsum(spec, Wi, A).reshape(wl_ * A.shape[0], d, wr * A.shape[2]))
        return out
    monkeypatch.setattr(P, "mpo_apply", mixed)
    assert _mpo_gap() > 1e-3
