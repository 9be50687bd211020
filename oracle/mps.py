"""MPS construction, environments and effective Hamiltonians (Sec. II.A).

TEST INFRASTRUCTURE (oracle); see the package docstring.

Index conventions: site tensor A[l, s, r]; MPO W[w, w', s', s] (s' is the bra
index); left environment L[l', w, l] and right environment R[r', w, r] with the
primed (bra) index first.  L of site i contracts sites < i (h[1:i-1] of
Eq. tdvp1_h1i), R of site i contracts sites > i (h[i+1:N] of Eq. tdvp1_hiN).

Each contraction below is its definition written as one ``np.einsum``.  numpy's
default path search refuses any intermediate larger than the largest operand and
then falls back to the naive loop over all eight indices (hours at D = 64); the
``_PATH`` setting lifts that cap so the same sum is evaluated pairwise.  The
pairing changes only the rounding order, not the result.
"""
from __future__ import annotations

import numpy as np

from .linalg import lq_rr

_PATH = ("greedy", 1e15)


def heff_apply(L, W, R, A):
    """H[i] C of Eq. tdvp2_C with H[i] from Eq. tdvp1_H.

    out[x,t,y] = sum_{w,v,a,s,b} L[x,w,a] W[w,v,t,s] A[a,s,b] R[y,v,b].
    """
    return np.einsum("xwa,wvts,asb,yvb->xty", L, W, A, R, optimize=_PATH)


def h0_apply(L, R, D):
    """Zero-site Hamiltonian of Eq. tdvp2_D: out[x,y] = sum_{w,a,b} L[x,w,a] D[a,b] R[y,w,b]."""
    return np.einsum("xwa,ab,ywb->xy", L, D, R, optimize=_PATH)


def env_left(L, A, W):
    """h[1:i] from h[1:i-1] and site i (Eq. tdvp1_h1i with Eq. tdvp1_h).

    Lnew[p,v,q] = sum_{x,w,y,t,s} L[x,w,y] conj(A[x,t,p]) W[w,v,t,s] A[y,s,q].
    """
    return np.einsum("xwy,xtp,wvts,ysq->pvq", L, A.conj(), W, A, optimize=_PATH)


def env_right(R, A, W):
    """h[i:N] from h[i+1:N] and site i (Eq. tdvp1_hiN with Eq. tdvp1_h).

    Rnew[p,w,q] = sum_{t,x,v,s,y} conj(A[p,t,x]) W[w,v,t,s] A[q,s,y] R[x,v,y].
    """
    return np.einsum("ptx,wvts,qsy,xvy->pwq", A.conj(), W, A, R, optimize=_PATH)


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

    Why r first: one-site TDVP-PS only moves the state inside the tangent space
    that these completion rows span.  Ordered s first, a site with Dl <= Dr gets
    only rows whose own level is the occupied one, the exciton-hopping direction is
    never in that space and the populations stay frozen at their start values;
    ordered r first, the rows are the single-site excitations that H reaches from
    the product state.  A CPU test holds the product start on the tiny chain to the
    exact state vector (max |dP| 1.0e-4 at D = 8, 7.9e-6 at D = 16 over 400 fs;
    0.53, the full transfer amplitude, with the s-first order).
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
    normalised to ||Psi|| = 1.  The carried tensor is rescaled to unit norm after each
    absorbed factor: the norm of a product of generic tensors grows or shrinks
    geometrically with the chain length and would leave the float64 range on long
    chains, while a positive scale changes neither the right-canonical factors (the
    LQ of s*C is (s*Dm) Qr) nor the normalised state.
    """
    mps = [np.array(t, dtype=complex) for t in tensors]
    for i in range(len(mps) - 1, 0, -1):
        Dl, d, Dr = mps[i].shape
        Dm, Qr = lq_rr(mps[i].reshape(Dl, d * Dr))
        mps[i] = Qr.reshape(Dl, d, Dr)
        mps[i - 1] = np.einsum("asb,bc->asc", mps[i - 1], Dm)
        mps[i - 1] = mps[i - 1] / np.linalg.norm(mps[i - 1])
    return mps


def mps_to_dense(mps):
    """Full state vector (tiny chains only)."""
    psi = mps[0].reshape(mps[0].shape[1], mps[0].shape[2])
    for A in mps[1:]:
        psi = np.einsum("xa,asb->xsb", psi, A).reshape(-1, A.shape[2])
    return psi.reshape(-1)
