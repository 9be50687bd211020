"""TDVP-MU: time-dependent variational principle in a fixed (left-canonical) gauge with the
matrix-unfolding regularisation, integrated by the second-order constant-mean-field scheme
(Sec. II.A.2, TDVP-MU paragraph; Eq. tdvp1_C, tdvp1_L, tdvp1_mu_rcano, tdvp1_mu_L, reg2).

TEST INFRASTRUCTURE (oracle); see the package docstring.

State: sites 1..N-1 left-canonical (L_i), the last site the coefficient tensor C_N.  Equations
of motion (Eq. tdvp1_C, Eq. tdvp1_L with the unfolding of Eq. tdvp1_mu_L):

    i dC_N/dt = H[N] C_N
    i dL_i/dt = (1 - p[i]) Hr[i](L_i U_i Lambda_i) Lambda~_i^-1 U_i^dag,      p[i] = L_i L_i^dag

where, for the bond after site i, the right part of the state (sites i+1..N) is written in an
orthonormal basis by moving the centre to site i+1 and decomposing it by SVD (Eq.
tdvp1_mu_rcano): |l_i> = sum_r U_{l r} Lambda_r |r_i>; Hr[i] is the one-site effective
Hamiltonian (Eq. tdvp1_H) with the left environment of the L's and the right environment of the
orthonormal |r_i> (the R tensors); and only the Lambda that multiplies the inverse is
regularised (Eq. reg2): Lambda~ = Lambda + eps^(1/2) exp(-Lambda / eps^(1/2)), eps = 1e-10.
(The product U^T U^* in the middle of Eq. tdvp1_mu_L is the identity and is contracted first.)

Constant mean field, second order, midpoint: the mean fields (the environments of every site,
U_i and Lambda_i) are built from the state at t, every L_i and C_N is integrated from t to
t + tau/2 with them held fixed, the mean fields are rebuilt from that midpoint state, and every
L_i and C_N is integrated again from t to t + tau with the midpoint fields.

Readings:
* with the mean fields fixed, the C_N equation is linear and is integrated by the Lanczos
  exponential of the one-site oracle; each L_i equation (nonlinear through p[i]) is integrated
  by Dormand-Prince RK45 (scipy ``solve_ivp``; rtol 1e-10, atol 1e-12 by default), the
  integrator the paper uses for VMF;
* the right decomposition is made once per mean-field evaluation by one SVD sweep from site N:
  the centre matrix at site j is SVD-decomposed, V^dag becomes the right-canonical R_j and
  U Lambda is carried into site j-1, so each bond's U, Lambda and the R tensors come from the
  same sweep;
* the start is left-canonicalised by the oracle's QR (Eq. QR) with the norm in C_N normalised
  to one.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp

from workloads import PHASE_PER_CM_FS
from .linalg import qr_rr, lanczos_expm
from .mps import heff_apply, env_left, env_right

EPS = 1e-10


def left_canonicalise(tensors):
    """Sites 1..N-1 left-canonical by QR from the left (Eq. QR), the norm of C_N set to one."""
    mps = [np.array(t, dtype=complex) for t in tensors]
    for i in range(len(mps) - 1):
        Dl, d, Dr = mps[i].shape
        Q, R = qr_rr(mps[i].reshape(Dl * d, Dr))
        mps[i] = Q.reshape(Dl, d, Dr)
        mps[i + 1] = np.einsum("ab,bsc->asc", R, mps[i + 1])
        mps[i + 1] = mps[i + 1] / np.linalg.norm(mps[i + 1])
    return mps


def regularise(lam, eps=EPS):
    """Eq. reg2: Lambda + eps^(1/2) exp(-Lambda / eps^(1/2))."""
    s = np.sqrt(eps)
    return lam + s * np.exp(-lam / s)


def mean_fields(W, mps):
    """Environments and unfoldings of the state (Eq. tdvp1_h1i, Eq. tdvp1_mu_rcano).

    Returns (Lenv, Renv, U, Lam): Lenv[i] from L_1..L_{i-1}; for i < N-1, Renv[i] from the
    orthonormal right tensors of sites i+1..N and (U[i], Lam[i]) with
    |l_i> = sum_r U[i][l, r] Lam[i][r] |r_i>; Renv[N-1] is the trivial right end."""
    N = len(mps)
    one = np.ones((1, 1, 1), dtype=complex)
    Lenv = [None] * N
    Lenv[0] = one
    for i in range(N - 1):
        Lenv[i + 1] = env_left(Lenv[i], mps[i], W[i])
    Renv = [None] * N
    U = [None] * N
    Lam = [None] * N
    Renv[N - 1] = one
    carry = None
    for j in range(N - 1, 0, -1):
        M = mps[j] if carry is None else np.einsum("asb,bc->asc", mps[j], carry)
        Dl, d, Dr = M.shape
        u, s, vh = np.linalg.svd(M.reshape(Dl, d * Dr), full_matrices=False)
        Rj = vh.reshape(-1, d, Dr)
        U[j - 1], Lam[j - 1] = u, s
        Renv[j - 1] = env_right(Renv[j], Rj, W[j])
        carry = u * s
    return Lenv, Renv, U, Lam


def site_derivative(W_i, Lenv_i, Renv_i, U_i, Lam_i, Li, eps=EPS):
    """dL_i/dt of Eq. tdvp1_mu_L for the left-canonical site tensor Li with the given fields."""
    Dl, d, Dr = Li.shape
    X = np.einsum("asb,br->asr", Li, U_i * Lam_i)
    Y = heff_apply(Lenv_i, W_i, Renv_i, X)
    Y = np.einsum("asr,r,lr->asl", Y, 1.0 / regularise(Lam_i, eps), U_i.conj())
    Lm = Li.reshape(Dl * d, Dr)
    Ym = Y.reshape(Dl * d, Dr)
    Ym = Ym - Lm @ (Lm.conj().T @ Ym)
    return (-1j * Ym).reshape(Dl, d, Dr)


def derivative(W, mps, eps=EPS):
    """The time derivative of every tensor at the state `mps` (fields from the same state)."""
    Lenv, Renv, U, Lam = mean_fields(W, mps)
    N = len(mps)
    out = [site_derivative(W[i], Lenv[i], Renv[i], U[i], Lam[i], mps[i], eps) for i in range(N - 1)]
    out.append(-1j * heff_apply(Lenv[N - 1], W[N - 1], Renv[N - 1], mps[N - 1]))
    return out


def _propagate(W, start, fields, t, eps, rtol, atol, tol, kmax):
    """Every L_i and C_N integrated from `start` over t (in cm) with the mean fields fixed."""
    Lenv, Renv, U, Lam = fields
    N = len(start)
    out = []
    for i in range(N - 1):
        shape = start[i].shape

        def rhs(_, y, i=i, shape=shape):
            return site_derivative(W[i], Lenv[i], Renv[i], U[i], Lam[i], y.reshape(shape), eps).ravel()
        sol = solve_ivp(rhs, (0.0, t), start[i].ravel(), method="RK45", rtol=rtol, atol=atol)
        if not sol.success:
            raise RuntimeError(f"RK45 failed at site {i}: {sol.message}")
        out.append(sol.y[:, -1].reshape(shape))
    C = lanczos_expm(lambda x: heff_apply(Lenv[N - 1], W[N - 1], Renv[N - 1], x), start[N - 1], -1j * t,
                     tol, kmax)
    out.append(C)
    return out


def tdvp_mu_step(W, mps, dt_fs, eps=EPS, rtol=1e-10, atol=1e-12, tol=1e-12, kmax=60):
    """One second-order CMF step (midpoint mean fields) of TDVP-MU over dt."""
    tau = dt_fs * PHASE_PER_CM_FS
    half = _propagate(W, mps, mean_fields(W, mps), tau / 2, eps, rtol, atol, tol, kmax)
    return _propagate(W, mps, mean_fields(W, half), tau, eps, rtol, atol, tol, kmax)
