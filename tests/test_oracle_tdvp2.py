"""Pins of the two-site TDVP-PS oracle (end of Sec. II.A.2; Eq. SVD for the split); CPU only.

- the two-site effective Hamiltonian equals P^H H P for the pair projector built densely from the
  MPS bases (dense H term by term, no environments);
- at maximal bond dimension from a random full-rank start the step is exact (the manifold is the
  whole space), to 1e-12 over ten steps;
- from a random bond-2 start the bonds grow to their maximum in the first step and the error at
  fixed time falls as dt^2 (symmetric split);
- without truncation norm and <H> are conserved; with a bond cap the bonds stay at the cap and
  the norm only falls;
- from the Hartree product start nothing grows on this chain: the hopping joins electronic sites
  three chain positions apart, so no two-site update of a product state entangles them (the
  reason for the paper's P&C-RK4 warm-up);
- planted mistakes (backward sign, a skipped backward step, the singular values kept on the wrong
  side of a split) each break the exactness pin.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import build_mpo, mps_to_dense, canonicalize_right, product_mps, qr_rr, env_left, env_right
from oracle.dense import hamiltonian_kron, propagate_exact, product_state
import oracle.tdvp2 as T2
from oracle.tdvp2 import tdvp2_step, heff2_apply


def _centre_at(mps, i):
    out = [A.copy() for A in mps]
    for j in range(i):
        Dl, d, Dr = out[j].shape
        Q, Rm = qr_rr(out[j].reshape(Dl * d, Dr))
        out[j] = Q.reshape(Dl, d, Dr)
        out[j + 1] = np.einsum("ab,bsc->asc", Rm, out[j + 1])
    return out


def test_two_site_heff_equals_dense_pair_projection():
    p = wl.tiny_chain()
    d = p.phys_dims()
    W = build_mpo(p)
    H = hamiltonian_kron(p)
    mps = _centre_at(canonicalize_right(wl.random_mps_tensors(d, 3, seed=8)), 2)
    i = 2
    UL = np.ones((1, 1))
    for A in mps[:i]:
        UL = np.einsum("xa,asb->xsb", UL, A).reshape(-1, A.shape[2])
    UR = np.ones((1, 1))
    for A in mps[:i + 1:-1]:
        UR = np.einsum("asb,bx->asx", A, UR).reshape(A.shape[0], -1)
    P = np.kron(np.kron(UL, np.eye(d[i] * d[i + 1])), UR.T)
    Hd = P.conj().T @ H @ P
    L = np.ones((1, 1, 1), complex)
    for j in range(i):
        L = env_left(L, mps[j], W[j])
    R = np.ones((1, 1, 1), complex)
    for j in range(len(d) - 1, i + 1, -1):
        R = env_right(R, mps[j], W[j])
    shape = (mps[i].shape[0], d[i], d[i + 1], mps[i + 1].shape[2])
    x = np.random.default_rng(3).normal(size=shape) + 1j * np.random.default_rng(4).normal(size=shape)
    got = heff2_apply(L, W[i], W[i + 1], R, x).reshape(-1)
    assert np.abs(got - Hd @ x.reshape(-1)).max() <= 1e-10 * np.abs(Hd).max()


def _exact_gap(steps=10, D0=32, dt=10.0):
    p = wl.tiny_chain()
    W = build_mpo(p)
    s = canonicalize_right(wl.random_mps_tensors(p.phys_dims(), D0, seed=9))
    ex = propagate_exact(hamiltonian_kron(p), mps_to_dense(s), dt * np.arange(1, steps + 1))
    worst = 0.0
    for k in range(steps):
        s = T2.tdvp2_step(W, s, dt, 1000)
        worst = max(worst, np.linalg.norm(mps_to_dense(s) - ex[k]))
    return worst, s


def test_full_bond_dimension_is_exact():
    worst, _ = _exact_gap()
    assert worst <= 1e-12


def test_bonds_grow_and_error_is_second_order():
    p = wl.tiny_chain()
    W = build_mpo(p)
    t = canonicalize_right(wl.random_mps_tensors(p.phys_dims(), 2, seed=9))
    ref = propagate_exact(hamiltonian_kron(p), mps_to_dense(t), [40.0])[0]
    errs = []
    for dt in (10.0, 5.0, 2.5):
        s = t
        for _ in range(int(40.0 / dt)):
            s = tdvp2_step(W, s, dt, 1000)
        assert [A.shape[2] for A in s] == [2, 8, 32, 16, 4, 1]
        errs.append(np.linalg.norm(mps_to_dense(s) - ref))
    for a, b in zip(errs, errs[1:]):
        assert 3.0 <= a / b <= 6.0, errs


def test_conservation_and_truncation():
    p = wl.tiny_chain()
    W = build_mpo(p)
    H = hamiltonian_kron(p)
    t = canonicalize_right(wl.random_mps_tensors(p.phys_dims(), 2, seed=9))

    def energy(v):
        return (v.conj() @ H @ v).real / (v.conj() @ v).real
    e0 = energy(mps_to_dense(t))
    s = t
    for _ in range(4):
        s = tdvp2_step(W, s, 10.0, 1000)
        v = mps_to_dense(s)
        assert abs(np.linalg.norm(v) - 1.0) <= 1e-12
        assert abs(energy(v) - e0) <= 1e-10 * max(1.0, abs(e0))
    s, prev = t, 1.0 + 1e-15
    for _ in range(4):
        s = tdvp2_step(W, s, 10.0, 4)
        n = np.linalg.norm(mps_to_dense(s))
        assert max(A.shape[2] for A in s) == 4 and n <= prev
        prev = n
    assert prev < 1.0 - 1e-4


def test_product_start_stays_a_product_on_this_chain():
    p = wl.tiny_chain()
    W = build_mpo(p)
    s = product_mps(p.phys_dims(), [1] * (len(p.phys_dims()) + 1), p.occupied())
    for _ in range(3):
        s = tdvp2_step(W, s, 10.0, 1000)
    assert all(A.shape[2] == 1 for A in s)
    assert np.linalg.norm(mps_to_dense(s) - propagate_exact(hamiltonian_kron(p), product_state(p), [30.0])[0]) > 0.1


# ---------------------------------------------------------------- planted mistakes (CPU)

def test_backward_sign_flip_is_caught(monkeypatch):
    orig = T2.lanczos_expm

    def flipped(matvec, v, z, *a, **k):
        if v.ndim == 3:                       # the one-site backward step
            z = -z
        return orig(matvec, v, z, *a, **k)
    monkeypatch.setattr(T2, "lanczos_expm", flipped)
    assert _exact_gap(steps=2)[0] > 1e-4


def test_skipped_backward_step_is_caught(monkeypatch):
    orig = T2.lanczos_expm
    monkeypatch.setattr(T2, "lanczos_expm",
                        lambda matvec, v, z, *a, **k: v if v.ndim == 3 else orig(matvec, v, z, *a, **k))
    assert _exact_gap(steps=2)[0] > 1e-4


def test_singular_values_on_the_wrong_side_are_caught(monkeypatch):
    orig = T2.truncated_svd

    def wrong_side(M, D, zeta=0.0):
        U, S, Vh = orig(M, D, zeta)
        return U * S, np.ones_like(S), Vh        # U Lambda as the "isometry", V^dag alone
    monkeypatch.setattr(T2, "truncated_svd", wrong_side)
    assert _exact_gap(steps=2)[0] > 1e-4
