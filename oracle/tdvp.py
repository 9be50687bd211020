"""One-site TDVP projector-splitting time step and observables (Sec. II.A.2, III.A).

TEST INFRASTRUCTURE (oracle); see the package docstring.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

from workloads import bond_dims, PHASE_PER_CM_FS
from .linalg import qr_rr, lq_rr, lanczos_expm
from .mpo import build_mpo, local_operators
from .mps import (heff_apply, h0_apply, env_left, env_right, product_mps, canonicalize_right)


@dataclass
class TDVPState:
    """MPS with its centre at site 0 plus every right environment.

    ``mps[0]`` is the centre C; ``mps[1:]`` are right-canonical.  ``Lenv[i]`` /
    ``Renv[i]`` are the environments of site i (sites < i / sites > i).
    """
    W: list
    mps: list
    Lenv: list
    Renv: list
    kinds: list
    t_fs: float = 0.0
    krylov_dims: list = field(default_factory=list)

    @classmethod
    def start(cls, params, D=None, tensors=None):
        """Product start at bond dim D (Sec. II.C) or explicit tensors (right-canonicalised)."""
        W = build_mpo(params)
        d = params.phys_dims()
        if tensors is None:
            mps = product_mps(d, bond_dims(d, D), params.occupied())
        else:
            mps = canonicalize_right(tensors)
        N = len(mps)
        Lenv = [None] * N
        Renv = [None] * N
        Lenv[0] = np.ones((1, 1, 1), dtype=complex)
        Renv[N - 1] = np.ones((1, 1, 1), dtype=complex)
        for i in range(N - 1, 0, -1):
            Renv[i - 1] = env_right(Renv[i], mps[i], W[i])
        kinds = [k for k, _, _ in params.chain()]
        return cls(W=W, mps=mps, Lenv=Lenv, Renv=Renv, kinds=kinds)


def tdvp_ps_step(st: TDVPState, dt_fs: float, tol=1e-12, kmax=60, rank_rtol=1e-13):
    """Advance by dt with the symmetric second-order split of Eq. ps_trotter.

    Left-to-right half sweep with tau/2 (Eq. tdvp2_C forward, Eq. QR, Eq. tdvp2_D
    backward with +i tau/2, C_{i+1} = D_i R_{i+1}), the last site with the full tau
    (one exponential, reading of the middle factor of Eq. ps_trotter), then the
    mirror right-to-left half sweep with LQ, ending with the forward step of site 1.
    H is in cm^-1 and dt in fs, so the exponent is -i * (2 pi c) * dt * H.
    ``rank_rtol`` is the relative rank threshold of the gauge-shift QR (see qr_rr).
    """
    tau = dt_fs * PHASE_PER_CM_FS
    A, W, L, R = st.mps, st.W, st.Lenv, st.Renv
    N = len(A)
    kd = st.krylov_dims

    def fwd(i, t):
        A[i] = lanczos_expm(lambda x: heff_apply(L[i], W[i], R[i], x), A[i], -1j * t, tol, kmax,
                            stats=kd)

    for i in range(N - 1):
        fwd(i, tau / 2)
        Dl, d, Dr = A[i].shape
        Q, Rm = qr_rr(A[i].reshape(Dl * d, Dr), rank_rtol)
        A[i] = Q.reshape(Dl, d, Dr)
        L[i + 1] = env_left(L[i], A[i], W[i])
        Rm = lanczos_expm(lambda x: h0_apply(L[i + 1], R[i], x), Rm, 1j * tau / 2, tol, kmax, stats=kd)
        A[i + 1] = np.einsum("ab,bsc->asc", Rm, A[i + 1])
    fwd(N - 1, tau)
    for i in range(N - 1, 0, -1):
        Dl, d, Dr = A[i].shape
        Dm, Qr = lq_rr(A[i].reshape(Dl, d * Dr), rank_rtol)
        A[i] = Qr.reshape(Dl, d, Dr)
        R[i - 1] = env_right(R[i], A[i], W[i])
        Dm = lanczos_expm(lambda x: h0_apply(L[i], R[i - 1], x), Dm, 1j * tau / 2, tol, kmax, stats=kd)
        A[i - 1] = np.einsum("asb,bc->asc", A[i - 1], Dm)
        fwd(i - 1, tau / 2)
    st.t_fs += dt_fs
    return st


def _expect_local(mps, ops_at):
    """<Psi| prod_i O_i |Psi> by a left-to-right transfer pass (O_i = identity if absent)."""
    E = np.ones((1, 1), dtype=complex)
    for i, A in enumerate(mps):
        O = ops_at.get(i)
        B = A if O is None else np.tensordot(O, A, axes=(1, 1)).transpose(1, 0, 2)
        T = np.tensordot(E, B, axes=(1, 0))                     # [x, t, q]
        E = np.tensordot(A.conj(), T, axes=([0, 1], [0, 1]))   # [p, q]
    return E[0, 0]


def norm(st: TDVPState):
    return float(np.sqrt(abs(_expect_local(st.mps, {}))))


def populations(st: TDVPState, params):
    """P^(n) = <n_n>/<Psi|Psi> for every electronic site label n (Eq. error)."""
    nrm2 = _expect_local(st.mps, {}).real
    chain = params.chain()
    out = np.zeros(params.n_el)
    nop = local_operators("el", 2)["n"]
    for i, (kind, m, _) in enumerate(chain):
        if kind == "el":
            out[m] = _expect_local(st.mps, {i: nop}).real / nrm2
    return out


def energy(st: TDVPState):
    """<Psi|H|Psi>/<Psi|Psi> by contracting the whole MPO (independent of stored envs)."""
    E = np.ones((1, 1, 1), dtype=complex)
    for A, W in zip(st.mps, st.W):
        E = env_left(E, A, W)
    return float((E[0, 0, 0] / _expect_local(st.mps, {})).real)


def mean_cumulative_deviation(t, P, Pref):
    """error(t) of Eq. error at the last time of the grid, trapezoid quadrature.

    ``P`` and ``Pref`` are [n_times, n_el] populations on the grid ``t`` (t[0] = 0).
    """
    t = np.asarray(t, float)
    dev = np.abs(np.asarray(P) - np.asarray(Pref)).sum(axis=1)
    integral = np.sum(0.5 * (dev[1:] + dev[:-1]) * np.diff(t))
    n_el = np.asarray(P).shape[1]
    return float(integral / (n_el * t[-1]))
