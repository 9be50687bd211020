"""Pins of the TDVP-MU (CMF) oracle (Sec. II.A.2 TDVP-MU; Eq. tdvp1_C, tdvp1_L, tdvp1_mu_rcano,
tdvp1_mu_L, reg2); CPU only.

- Dirac-Frenkel: the derivative of the state assembled from the equations of motion equals the
  orthogonal projection of -i H Psi onto the tangent space, the space built densely from its
  definition (every gauge-fixed variation of one left-canonical site, L^dag dL = 0, and every
  variation of C_N) with the Kronecker-built H; at maximal bond dimension it equals -i H Psi;
- Eq. reg2 in closed form, and a state with exactly zero singular values (the completed product
  start) gives a finite derivative only with the regularisation;
- CMF with midpoint mean fields converges at second order to the TDVP flow (one-site TDVP-PS at
  a 16x finer step integrates the same projected equation), and keeps the norm and the
  left-canonical condition;
- planted mistakes (the projector 1 - p dropped, Lambda left out of the unfolded input, U^T in
  place of U^dag, mean fields from the start instead of the midpoint) are each caught.
"""
import numpy as np
import pytest

import workloads as wl
from workloads import bond_dims
from oracle import build_mpo, mps_to_dense, product_mps, TDVPState, tdvp_ps_step
from oracle.dense import hamiltonian_kron
import oracle.tdvp_mu as MU
from oracle.tdvp_mu import left_canonicalise, derivative, regularise, tdvp_mu_step, EPS


def _dense_derivative(W, s, eps=EPS):
    der = MU.derivative(W, s, eps)
    return sum(mps_to_dense(s[:i] + [der[i]] + s[i + 1:]) for i in range(len(s)))


def _tangent_projection(s, v):
    """Orthogonal projection of v onto the tangent space at the left-canonical MPS s."""
    N = len(s)
    cols = []
    for i in range(N):
        UL = np.ones((1, 1))
        for A in s[:i]:
            UL = np.einsum("xa,asb->xsb", UL, A).reshape(-1, A.shape[2])
        RS = np.ones((1, 1))
        for A in s[:i:-1]:
            RS = np.einsum("asb,bx->asx", A, RS).reshape(A.shape[0], -1)
        Dl, d, Dr = s[i].shape
        if i < N - 1:
            Lm = s[i].reshape(Dl * d, Dr)
            Pp = np.eye(Dl * d) - Lm @ Lm.conj().T        # variations with L^dag dL = 0
            for a in range(Dl * d):
                for b in range(Dr):
                    X = np.outer(Pp[:, a], np.eye(Dr)[b]).reshape(Dl, d, Dr)
                    cols.append(np.einsum("xa,asb,by->xsy", UL, X, RS).reshape(-1))
        else:
            for a in range(Dl * d):
                cols.append(np.kron(UL, np.eye(d)).reshape(-1, Dl * d)[:, a])
    u, sv, _ = np.linalg.svd(np.array(cols).T, full_matrices=False)
    Q = u[:, :int(np.sum(sv > 1e-10 * sv[0]))]
    return Q @ (Q.conj().T @ v)


@pytest.mark.parametrize("D,seed", [(3, 9), (4, 9), (4, 21)])
def test_derivative_is_the_tangent_space_projection(D, seed):
    p = wl.tiny_chain()
    W = build_mpo(p)
    H = hamiltonian_kron(p)
    s = left_canonicalise(wl.random_mps_tensors(p.phys_dims(), D, seed=seed))
    psi = mps_to_dense(s)
    ref = _tangent_projection(s, -1j * H @ psi)
    got = _dense_derivative(W, s)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(got + 1j * H @ psi).max() > 1e-3 * np.abs(H @ psi).max()   # truncated: a real projection


def test_derivative_at_maximal_bond_dimension_is_the_schroedinger_rhs():
    p = wl.tiny_chain()
    W = build_mpo(p)
    H = hamiltonian_kron(p)
    s = left_canonicalise(wl.random_mps_tensors(p.phys_dims(), 32, seed=9))
    psi = mps_to_dense(s)
    assert np.abs(_dense_derivative(W, s) + 1j * H @ psi).max() <= 1e-12 * np.abs(H @ psi).max()


def test_regularisation_closed_form_and_zero_singular_values():
    s = np.sqrt(EPS)
    lam = np.array([0.0, s, 10 * s, 1e-2, 1.0])
    reg = regularise(lam)
    assert reg[0] == s and abs(reg[1] - s * (1 + np.exp(-1))) <= 1e-20
    assert np.all(np.diff(reg) > 0) and abs(reg[-1] - 1.0) <= 1e-15 and abs(reg[3] - 1e-2) <= 1e-15
    # the product start completed at D = 4 has exactly zero singular values on its bonds
    p = wl.tiny_chain()
    W = build_mpo(p)
    d = p.phys_dims()
    st = left_canonicalise(product_mps(d, bond_dims(d, 4), p.occupied()))
    _, _, _, Lam = MU.mean_fields(W, st)
    assert min(float(x.min()) for x in Lam[:-1]) == 0.0
    assert all(np.all(np.isfinite(x)) for x in derivative(W, st))
    with np.errstate(all="ignore"):
        bad = derivative(W, st, eps=0.0)
    assert not all(np.all(np.isfinite(x)) for x in bad)


def _cmf_errors(steps_dt=(10.0, 5.0, 2.5), T=40.0):
    p = wl.tiny_chain()
    W = build_mpo(p)
    tens = wl.random_mps_tensors(p.phys_dims(), 4, seed=9)
    st = TDVPState.start(p, tensors=tens)
    for _ in range(64):
        tdvp_ps_step(st, T / 64)
    ref = mps_to_dense(st.mps)
    errs, last = [], None
    for dt in steps_dt:
        x = left_canonicalise(tens)
        for _ in range(int(round(T / dt))):
            x = MU.tdvp_mu_step(W, x, dt)
        errs.append(np.linalg.norm(mps_to_dense(x) - ref))
        last = x
    return errs, last


def test_cmf_is_second_order_and_keeps_norm_and_gauge():
    errs, x = _cmf_errors()
    for a, b in zip(errs, errs[1:]):
        assert 3.0 <= a / b <= 6.0, errs
    assert abs(np.linalg.norm(mps_to_dense(x)) - 1.0) <= 1e-10
    for A in x[:-1]:
        M = A.reshape(-1, A.shape[2])
        assert np.abs(M.conj().T @ M - np.eye(A.shape[2])).max() <= 1e-8


# ---------------------------------------------------------------- planted mistakes (CPU)

def _projection_gap():
    p = wl.tiny_chain()
    W = build_mpo(p)
    s = left_canonicalise(wl.random_mps_tensors(p.phys_dims(), 4, seed=9))
    ref = _tangent_projection(s, -1j * hamiltonian_kron(p) @ mps_to_dense(s))
    return np.abs(_dense_derivative(W, s) - ref).max() / np.abs(ref).max()


def test_pins_are_quiet_without_a_mistake():
    assert _projection_gap() < 1e-12


def test_dropped_projector_is_caught(monkeypatch):
    def no_projector(W_i, Lenv_i, Renv_i, U_i, Lam_i, Li, eps=EPS):
        X = np.einsum("asb,br->asr", Li, U_i * Lam_i)
        Y = MU.heff_apply(Lenv_i, W_i, Renv_i, X)
        return -1j * np.einsum("asr,r,lr->asl", Y, 1.0 / regularise(Lam_i, eps), U_i.conj())
    monkeypatch.setattr(MU, "site_derivative", no_projector)
    assert _projection_gap() > 1e-3


def test_lambda_left_out_of_the_input_is_caught(monkeypatch):
    def no_lambda(W_i, Lenv_i, Renv_i, U_i, Lam_i, Li, eps=EPS):
        Dl, d, Dr = Li.shape
        X = np.einsum("asb,br->asr", Li, U_i)                  # L U instead of L U Lambda
        Y = MU.heff_apply(Lenv_i, W_i, Renv_i, X)
        Ym = np.einsum("asr,r,lr->asl", Y, 1.0 / regularise(Lam_i, eps), U_i.conj()).reshape(Dl * d, Dr)
        Lm = Li.reshape(Dl * d, Dr)
        return (-1j * (Ym - Lm @ (Lm.conj().T @ Ym))).reshape(Dl, d, Dr)
    monkeypatch.setattr(MU, "site_derivative", no_lambda)
    assert _projection_gap() > 1e-3


def test_transpose_in_place_of_adjoint_is_caught(monkeypatch):
    orig = MU.mean_fields

    def conj_u(W, mps):
        Lenv, Renv, U, Lam = orig(W, mps)
        return Lenv, Renv, [None if u is None else u.conj() for u in U], Lam
    monkeypatch.setattr(MU, "mean_fields", conj_u)
    assert _projection_gap() > 1e-3


def test_start_fields_instead_of_midpoint_fields_are_caught(monkeypatch):
    def first_order(W, mps, dt_fs, eps=EPS, rtol=1e-10, atol=1e-12, tol=1e-12, kmax=60):
        tau = dt_fs * MU.PHASE_PER_CM_FS
        return MU._propagate(W, mps, MU.mean_fields(W, mps), tau, eps, rtol, atol, tol, kmax)
    monkeypatch.setattr(MU, "tdvp_mu_step", first_order)
    errs, _ = _cmf_errors()
    assert errs[1] / errs[2] < 3.0, errs
