"""MPS construction, environments and effective Hamiltonians (Sec. II.A).

TEST INFRASTRUCTURE (oracle); see the package docstring.

Index conventions: site tensor A[l, s, r]; MPO W[w, w', s', s] (s' is the bra
index); left environment L[l', w, l] and right environment R[r', w, r] with the
primed (bra) index first.  L of site i contracts sites < i (h[1:i-1] of
Eq. tdvp1_h1i), R of site i contracts sites > i (h[i+1:N] of Eq. tdvp1_hiN).
"""
from __future__ import annotations

import numpy as np

from .linalg import lq_rr


def heff_apply(L, W, R, A):
    """H[i] C of Eq. tdvp2_C with H[i] from Eq. tdvp1_H, contracted stage by stage.

    T1[x,w,s,b] = sum_a L[x,w,a] A[a,s,b]; T2 = sum_{w,s} T1 W[w,v,t,s];
    out[x,t,y] = sum_{v,b} T2[x,b,v,t] R[y,v,b].
    """
    T1 = np.tensordot(L, A, axes=(2, 0))                    # [x, w, s, b]
    T2 = np.tensordot(T1, W, axes=([1, 2], [0, 3]))         # [x, b, v, t]
    return np.tensordot(T2, R, axes=([1, 2], [2, 1]))       # [x, t, y]


def h0_apply(L, R, D):
    """Zero-site Hamiltonian of Eq. tdvp2_D: out[x,y] = sum_{w,a,b} L[x,w,a] D[a,b] R[y,w,b]."""
    T = np.tensordot(L, D, axes=(2, 0))                     # [x, w, b]
    return np.tensordot(T, R, axes=([1, 2], [1, 2]))        # [x, y]


def env_left(L, A, W):
    """h[1:i] from h[1:i-1] and site i (Eq. tdvp1_h1i with Eq. tdvp1_h).

    Lnew[p,v,q] = sum L[x,w,y] conj(A[x,t,p]) W[w,v,t,s] A[y,s,q].
    """
    T1 = np.tensordot(L, A, axes=(2, 0))                    # [x, w, s, q]
    T2 = np.tensordot(T1, W, axes=([1, 2], [0, 3]))         # [x, q, v, t]
    out = np.tensordot(A.conj(), T2, axes=([0, 1], [0, 3])) # [p, q, v]
    return out.transpose(0, 2, 1)


def env_right(R, A, W):
    """h[i:N] from h[i+1:N] and site i (Eq. tdvp1_hiN with Eq. tdvp1_h).

    Rnew[p,w,q] = sum conj(A[p,t,x]) W[w,v,t,s] A[q,s,y] R[x,v,y].
    """
    T1 = np.tensordot(A, R, axes=(2, 2))                    # [q, s, x, v]
    T2 = np.tensordot(T1, W, axes=([1, 3], [3, 1]))         # [q, x, w, t]
    out = np.tensordot(A.conj(), T2, axes=([1, 2], [3, 1])) # [p, q, w]
    return out.transpose(0, 2, 1)


def product_mps(d, bd, occ):
    """Right-canonical MPS of a product state at bond dims ``bd`` (Sec. II.C start).

    Reading of the basis completion the paper asks for (Sec. II.A.2, end of
    TDVP-PS; Sec. II.C): row 0 of site i (viewed as a Dl x (d*Dr) matrix) is the
    occupied path, A[0, occ_i, 0] = 1; row j >= 1 is the standard basis vector at
    the j-th position (s, r) other than (occ_i, 0), positions ordered by r first
    and s second, so that the local excitations of the occupied right path come
    first.
    Distinct standard basis rows are orthonormal, so every site is
    right-canonical (Eq. rcanon) and the state is the product state.
    """
    mps = []
    for i, di in enumerate(d):
        Dl, Dr = bd[i], bd[i + 1]
        A = np.zeros((Dl, di, Dr), dtype=complex)
        A[0, occ[i], 0] = 1.0
        j = 1
        for r in range(Dr):
            for s in range(di):
                if j >= Dl:
                    break
                if s == occ[i] and r == 0:
                    continue
                A[j, s, r] = 1.0
                j += 1
        mps.append(A)
    return mps


def canonicalize_right(tensors):
    """Right-canonical form by LQ from the last site to the first (Eq. QR, "RQ").

    Returns new tensors with sites 1..N-1 right-canonical and the centre at site 0,
    normalised to ||Psi|| = 1.
    """
    mps = [np.array(t, dtype=complex) for t in tensors]
    for i in range(len(mps) - 1, 0, -1):
        Dl, d, Dr = mps[i].shape
        Dm, Qr = lq_rr(mps[i].reshape(Dl, d * Dr))
        mps[i] = Qr.reshape(Dl, d, Dr)
        mps[i - 1] = np.einsum("asb,bc->asc", mps[i - 1], Dm)
    mps[0] = mps[0] / np.linalg.norm(mps[0])
    return mps


def mps_to_dense(mps):
    """Full state vector (tiny chains only)."""
    psi = mps[0].reshape(mps[0].shape[1], mps[0].shape[2])
    for A in mps[1:]:
        psi = np.einsum("xa,asb->xsb", psi, A).reshape(-1, A.shape[2])
    return psi.reshape(-1)
