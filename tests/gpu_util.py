"""Helpers shared by the GPU tests (CUDA path vs CPU oracle on the same seeded inputs)."""
import numpy as np
import pytest

import paper_1907_12044_b300 as pkg
from oracle import TDVPState, populations, energy, canonicalize_right, qr_rr, env_left, env_right


# Relative error bounds of one mixed-precision contraction, ||y - y_ref|| / ||y_ref||: 10 u of
# the operand format for the 4M modes (TF32 u = 2^-11, BF16 u = 2^-8), 20 u for 3M (one more
# rounding per operand), 2e-5 for TF32x3 and 10 x 2^-16 for BF16x3 (compensated products).
U_TF32, U_BF16 = 2.0 ** -11, 2.0 ** -8
MIXED_TOL = {pkg.PREC_TF32: 10 * U_TF32, pkg.PREC_TF32X3: 2e-5, pkg.PREC_BF16: 10 * U_BF16,
             pkg.PREC_BF16X3: 10 * 2.0 ** -16, pkg.PREC_TF32_3M: 20 * U_TF32, pkg.PREC_BF16_3M: 20 * U_BF16}
PREC_NAME = {pkg.PREC_TF32: "TF32", pkg.PREC_TF32X3: "TF32x3", pkg.PREC_BF16: "BF16",
             pkg.PREC_BF16X3: "BF16x3", pkg.PREC_TF32_3M: "TF32-3M", pkg.PREC_BF16_3M: "BF16-3M"}


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def engine_for(params, D=None, tensors=None, R=1, kmax=64):
    eng = pkg.Engine(n_realisations=R, kmax=kmax)
    for r in range(R):
        eng.build_mpo(r, params)
        if tensors is None:
            eng.init_mps(r, D, params.exciton_site)
        else:
            eng.init_mps_tensors(r, tensors)
    return eng


def oracle_centred(params, tensors, site):
    """The oracle's own mixed-canonical form of the start tensors with the centre at `site`, and
    the environments of that site, computed from the seeded tensors alone (nothing from the CUDA
    path): right-canonicalised by LQ (Eq. QR, right to left), then the centre moved right by QR
    shifts (Eq. QR), the environments built from these tensors (Eq. tdvp1_h1i, tdvp1_hiN).
    Returns (mps, W, L, R)."""
    W = TDVPState.start(params, D=1).W
    mps = canonicalize_right(tensors)
    for i in range(site):
        Dl, d, Dr = mps[i].shape
        Q, Rm = qr_rr(mps[i].reshape(Dl * d, Dr))
        mps[i] = Q.reshape(Dl, d, Dr)
        mps[i + 1] = np.einsum("ab,bsc->asc", Rm, mps[i + 1])
    L = np.ones((1, 1, 1), complex)
    for j in range(site):
        L = env_left(L, mps[j], W[j])
    R = np.ones((1, 1, 1), complex)
    for j in range(len(mps) - 1, site, -1):
        R = env_right(R, mps[j], W[j])
    return mps, W, L, R


def gauge_err(gpu_mps, mps, sites):
    """max over the given sites of max |A_gpu - A| / max |A| (the canonical form is unique for
    full-rank tensors: every QR factor has a positive diagonal)."""
    return max(float(np.abs(gpu_mps[i] - mps[i]).max() / np.abs(mps[i]).max()) for i in sites)


def rel_pop_err(P, Pref):
    return float(np.max(np.abs(np.asarray(P) - np.asarray(Pref))) / max(np.max(np.abs(Pref)), 1e-300))


def cluster_fits(C, m, n):
    """Whether an n x m QR fits the cluster kernel's shared memory with C CTAs (220 KiB each)."""
    ld = (-(-m // C)) | 1
    return C <= m and 16 * (n * ld + 2 * (n + 4) + 3 * n) + 8 * ld <= 220 * 1024


def debug_qr_or_rejected(eng, kernel, C):
    """debug_qr, or None after checking that a forced cluster size too small for C is rejected."""
    m, n = C.shape
    if kernel > 0 and not cluster_fits(kernel, m, n):
        with pytest.raises(pkg.TDVPError):
            eng.debug_qr(C)
        return None
    return eng.debug_qr(C)
