"""P&C-RK4: global propagation and compression of an MPS (Sec. II.A.1, Eq. RK4).

TEST INFRASTRUCTURE (oracle); see the package docstring.

The paper starts every TDVP run from a P&C-RK4 warm-up (Sec. II.C): the Hartree product
state is propagated with RK4 by whole-MPS operations, each followed by an SVD compression,
for 10 steps of 80 a.u. at M_max = 256, then compressed to the run's bond dimension M_S.
The operations, each written from its equation:

* MPO x MPS (Eq. mpo-apply): the site tensors of O|Psi> are the local contractions of the
  MPO tensor with the MPS tensor over the ket index; the bond becomes the pair (w, a);
* MPS + MPS (Eq. mps+mps): block-diagonal site tensors, a row block at the first site and
  a column block at the last;
* canonicalisation (Eq. QR, left to right) and compression by successive truncated SVDs
  from the last site to the first (Eq. SVD), keeping at each bond the M largest singular
  values (criterion i) and, optionally, only those above zeta (criterion ii);
* one RK4 step (Eq. RK4) for the time-independent Frenkel-Holstein H.

Readings (the paper does not fix them):
* every k_i and every stage state is compressed before it is used again (Sec. II.A.1 asks for
  a compression after each operation); the final combination Psi + tau/6 (k1 + 2 k2 + 2 k3 + k4) is formed as one
  block-diagonal sum of the five MPSs (Eq. mps+mps with five blocks) and compressed once;
* the canonicalisation QR is numpy's reduced QR (no rank decision: a bond larger than the
  rank of its matrix shrinks to min(rows, columns), and the SVD then drops the zero
  singular values);
* singular values at or below 1e-14 of the largest at a bond are dropped with the rest of
  the truncation (they carry no weight and only pad the bond);
* H is in cm^-1 and time in fs, as everywhere in the oracle; 80 a.u. of time is
  80 x 2.4188843e-2 fs (CODATA atomic unit of time).
"""
from __future__ import annotations

import numpy as np

from workloads import PHASE_PER_CM_FS
from .mpo import build_mpo
from .mps import product_mps

ATOMIC_TIME_FS = 2.4188843265857e-2      # CODATA 2018 atomic unit of time, in fs
SV_FLOOR = 1e-14


def mpo_apply(W, mps):
    """O|Psi> by Eq. mpo-apply: A'[(w,a), t, (v,b)] = sum_s W[w,v,t,s] A[a,s,b].

    W[i] has the layout (w_left, w_right, out, in); the new bond index is w-major."""
    out = []
    for Wi, A in zip(W, mps):
        wl, wr, d, _ = Wi.shape
        Dl, _, Dr = A.shape
        B = np.einsum("wvts,asb->watvb", Wi, A)
        out.append(B.reshape(wl * Dl, d, wr * Dr))
    return out


def mps_add(coefs, states):
    """sum_k c_k |Psi_k> by Eq. mps+mps, generalised to several terms.

    Site 1 is the row block [c_1 A_1, c_2 A_2, ...] (the coefficients sit there), sites
    2..N-1 are block diagonal, site N is the column block [A_1; A_2; ...]."""
    N = len(states[0])
    out = []
    for i in range(N):
        blocks = [s[i] for s in states]
        d = blocks[0].shape[1]
        Dl = 1 if i == 0 else sum(b.shape[0] for b in blocks)
        Dr = 1 if i == N - 1 else sum(b.shape[2] for b in blocks)
        T = np.zeros((Dl, d, Dr), dtype=complex)
        l0 = r0 = 0
        for c, b in zip(coefs, blocks):
            bl, _, br = b.shape
            if N == 1:
                T += c * b
                continue
            if i == 0:
                T[:, :, r0:r0 + br] = c * b
            elif i == N - 1:
                T[l0:l0 + bl, :, :] = b
            else:
                T[l0:l0 + bl, :, r0:r0 + br] = b
            l0 += bl
            r0 += br
        out.append(T)
    return out


def canonicalise_left(mps):
    """Left-canonical form with the centre at the last site, by QR from site 1 to N-1 (Eq. QR):
    C[(l s), r] = Q R, site i <- Q, site i+1 <- R A_{i+1}.  The norm stays in the last site."""
    out = [np.array(A, dtype=complex) for A in mps]
    for i in range(len(out) - 1):
        Dl, d, Dr = out[i].shape
        Q, R = np.linalg.qr(out[i].reshape(Dl * d, Dr))
        out[i] = Q.reshape(Dl, d, Q.shape[1])
        out[i + 1] = np.einsum("ab,bsc->asc", R, out[i + 1])
    return out


def svd_compress(mps, M, zeta=0.0):
    """Compression of a left-canonical MPS (centre at the last site) by successive truncated
    SVDs from site N to 2 (Eq. SVD, right-to-left form): C[l, (s r)] = U Lambda V^dag; site i
    keeps the rows of V^dag of the M largest singular values (criterion i), and with zeta > 0
    only those with Lambda_s > zeta ||Lambda|| (criterion ii, relative to the norm of the state
    so that it also applies to the unnormalised k_i); site i-1 absorbs U Lambda of the kept
    ones.  Returns a right-canonical MPS with the centre (and the norm) at the first site."""
    out = [np.array(A, dtype=complex) for A in mps]
    for i in range(len(out) - 1, 0, -1):
        Dl, d, Dr = out[i].shape
        U, S, Vh = np.linalg.svd(out[i].reshape(Dl, d * Dr), full_matrices=False)
        nrm = np.linalg.norm(S)
        keep = int(np.sum(S > max(zeta * nrm, SV_FLOOR * S[0]))) if S[0] > 0 else 0
        keep = max(1, min(M, keep))
        out[i] = Vh[:keep].reshape(keep, d, Dr)
        out[i - 1] = np.einsum("asb,bc->asc", out[i - 1], U[:, :keep] * S[:keep])
    return out


def compress(mps, M, zeta=0.0):
    """Canonicalisation followed by compression: the sum or MPO product is not canonical, and
    Sec. II.A.1 canonicalises it before the SVD sweep."""
    return svd_compress(canonicalise_left(mps), M, zeta)


def rk4_step(W, psi, dt_fs, M, zeta=0.0):
    """One P&C-RK4 step of Eq. RK4 for the time-independent H of the MPO W, every operation
    followed by a compression to at most M (the readings in the module docstring).  The
    derivative is -i H Psi with H in cm^-1, so the step is h = dt * 2 pi c in cm."""
    h = dt_fs * PHASE_PER_CM_FS

    def deriv(state):
        return compress(mps_add([-1j], [mpo_apply(W, state)]), M, zeta)

    k1 = deriv(psi)
    k2 = deriv(compress(mps_add([1.0, h / 2], [psi, k1]), M, zeta))
    k3 = deriv(compress(mps_add([1.0, h / 2], [psi, k2]), M, zeta))
    k4 = deriv(compress(mps_add([1.0, h], [psi, k3]), M, zeta))
    return compress(mps_add([1.0, h / 6, h / 3, h / 3, h / 6], [psi, k1, k2, k3, k4]), M, zeta)


def warmup(params, M_S, steps=10, dt_au=80.0, M_max=256, zeta=0.0):
    """The paper's warm-up (Sec. II.C): the Hartree product start (exciton on one site, every
    mode in its ground level) propagated by `steps` P&C-RK4 steps of dt_au atomic units at
    M_max, then compressed to M_S.  Returns right-canonical tensors with the centre at site 1
    (the norm, 1 up to the RK4 error, is left in the centre)."""
    W = build_mpo(params)
    d = params.phys_dims()
    psi = product_mps(d, [1] * (len(d) + 1), params.occupied())
    for _ in range(steps):
        psi = rk4_step(W, psi, dt_au * ATOMIC_TIME_FS, M_max, zeta)
    return compress(psi, M_S)
