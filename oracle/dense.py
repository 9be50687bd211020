"""Dense tiny-system references used to pin the oracle (state vectors, <= ~4096 dims).

TEST INFRASTRUCTURE (oracle); see the package docstring.
"""
from __future__ import annotations

from functools import reduce
import numpy as np
import scipy.linalg as sla

from workloads import PHASE_PER_CM_FS, bond_dims
from .linalg import qr_rr, lq_rr
from .mpo import local_operators


def _embed(op, i, d):
    mats = [np.eye(x) for x in d]
    mats[i] = op
    return reduce(np.kron, mats)


def hamiltonian_kron(p):
    """Dense H of Eq. holstein from Kronecker products of the local operators.

    Written term by term from the second-quantised form, independently of the MPO.
    """
    chain = p.chain()
    d = p.phys_dims()
    dim = int(np.prod(d))
    H = np.zeros((dim, dim))
    el_pos = {m: i for i, (kind, m, _) in enumerate(chain) if kind == "el"}
    for m, i in el_pos.items():
        ops = local_operators("el", 2)
        H += (p.E[m] - p.energy_offset) * _embed(ops["n"], i, d)
    for m, i in el_pos.items():
        for n, j in el_pos.items():
            if m != n and p.J[m, n] != 0.0:
                cr = _embed(local_operators("el", 2)["cr"], i, d)
                an = _embed(local_operators("el", 2)["an"], j, d)
                H += p.J[m, n] * cr @ an
    for i, (kind, m, k) in enumerate(chain):
        if kind != "vib":
            continue
        ops = local_operators("vib", d[i])
        w, g = p.omega[m][k], p.g[m][k]
        H += w * _embed(ops["nb"], i, d)
        if p.include_zpe:
            H += 0.5 * w * np.eye(dim)
        nel = _embed(local_operators("el", 2)["n"], el_pos[m], d)
        H += g * w * _embed(ops["x"], i, d) @ nel
    return H


def product_state(p):
    d = p.phys_dims()
    occ = p.occupied()
    vecs = []
    for di, o in zip(d, occ):
        v = np.zeros(di)
        v[o] = 1.0
        vecs.append(v)
    return reduce(np.kron, vecs).astype(complex)


def propagate_exact(H, psi0, times_fs):
    """psi(t) = exp(-i 2 pi c t H) psi0 by full eigendecomposition."""
    lam, U = np.linalg.eigh(H)
    c0 = U.conj().T @ psi0
    return [U @ (np.exp(-1j * PHASE_PER_CM_FS * t * lam) * c0) for t in times_fs]


def populations_dense(psi, p):
    chain = p.chain()
    d = p.phys_dims()
    out = np.zeros(p.n_el)
    nrm2 = np.vdot(psi, psi).real
    for i, (kind, m, _) in enumerate(chain):
        if kind == "el":
            op = _embed(local_operators("el", 2)["n"], i, d)
            out[m] = np.vdot(psi, op @ psi).real / nrm2
    return out


def _basis_left(iso_list, d, i):
    """Dense isometry of the left renormalised basis |l_i[1:i]> from left-canonical tensors."""
    U = np.ones((1, 1), dtype=complex)
    for j in range(i):
        A = iso_list[j]
        Dl, dj, Dr = A.shape
        U = np.einsum("xa,asb->xsb", U, A).reshape(-1, Dr)
    return U


def _basis_right(iso_list, d, i):
    """Dense isometry of the right basis |r_i[i+1:N]> (rows of right-canonical tensors)."""
    N = len(iso_list)
    U = np.ones((1, 1), dtype=complex)
    for j in range(N - 1, i, -1):
        A = iso_list[j]
        Dl, dj, Dr = A.shape
        U = np.einsum("asb,bx->asx", A, U).reshape(Dl, -1)
    return U          # [D_i, prod right dims]


def projector_split_step(psi, p, mps, H, dt_fs):
    """One step of Eq. ps_trotter with every factor applied as a dense exponential.

    ``mps`` gives the current gauge (centre at site 0, right-canonical rest) and is
    updated along the way; the state is carried as a dense vector ``psi`` and every
    sub-step applies exp(-/+ i P H P tau') with P = P[1:i-1] (x) I_i (x) P[i+1:N]
    or P[1:i] (x) P[i+1:N] built densely from the current bases (Sec. II.A.2,
    TDVP-PS).  Only the QR gauge choice is shared with the oracle.
    """
    tau = dt_fs * PHASE_PER_CM_FS
    d = p.phys_dims()
    N = len(d)
    A = [x.copy() for x in mps]
    dims = [int(np.prod(d[:i])) for i in range(N + 1)]

    def site_proj(i):
        UL = _basis_left(A, d, i)                 # [prod d<i, Dl]
        UR = _basis_right(A, d, i)                # [Dr, prod d>i]
        return np.kron(np.kron(UL, np.eye(d[i])), UR.T)        # columns: (l, s, r)

    def bond_proj(i):
        UL = _basis_left(A, d, i + 1)             # [prod d<=i, Dl']
        UR = _basis_right(A, d, i)                # [Dr, prod d>i]
        return np.kron(UL, UR.T)

    def apply(Pcols, z):
        Heff = Pcols.conj().T @ H @ Pcols
        coef = Pcols.conj().T @ psi
        coef = sla.expm(z * Heff) @ coef
        return Pcols @ coef, coef

    for i in range(N - 1):
        P = site_proj(i)
        psi, c = apply(P, -1j * tau / 2)
        Dl, di, Dr = A[i].shape
        Q, Rm = qr_rr(c.reshape(Dl * di, Dr))
        A[i] = Q.reshape(Dl, di, Dr)
        P = bond_proj(i)
        psi, c = apply(P, 1j * tau / 2)
        Rm = c.reshape(A[i].shape[2], A[i + 1].shape[0])
        A[i + 1] = np.einsum("ab,bsc->asc", Rm, A[i + 1])
    P = site_proj(N - 1)
    psi, c = apply(P, -1j * tau)
    A[N - 1] = c.reshape(A[N - 1].shape)
    for i in range(N - 1, 0, -1):
        Dl, di, Dr = A[i].shape
        Dm, Qr = lq_rr(A[i].reshape(Dl, di * Dr))
        A[i] = Qr.reshape(Dl, di, Dr)
        P = bond_proj(i - 1)
        psi, c = apply(P, 1j * tau / 2)
        Dm = c.reshape(A[i - 1].shape[2], Dl)
        A[i - 1] = np.einsum("asb,bc->asc", A[i - 1], Dm)
        P = site_proj(i - 1)
        psi, c = apply(P, -1j * tau / 2)
        A[i - 1] = c.reshape(A[i - 1].shape)
    return psi, A
