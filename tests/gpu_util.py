"""Helpers shared by the GPU tests (CUDA path vs CPU oracle on the same seeded inputs)."""
import numpy as np
import pytest

import paper_1907_12044_b300 as pkg
from oracle import TDVPState, populations, energy


def engine_for(params, D=None, tensors=None, R=1, kmax=64):
    eng = pkg.Engine(n_realisations=R, kmax=kmax)
    for r in range(R):
        eng.build_mpo(r, params)
        if tensors is None:
            eng.init_mps(r, D, params.exciton_site)
        else:
            eng.init_mps_tensors(r, tensors)
    return eng


def oracle_from_gpu_tensors(params, mps):
    """Oracle state over the given (right-canonical, centre at 0) tensors, with oracle-built envs."""
    st = TDVPState.start(params, D=1)
    st.mps = [np.array(a) for a in mps]
    from oracle.mps import env_right
    N = len(st.mps)
    st.Renv = [None] * N
    st.Renv[N - 1] = np.ones((1, 1, 1), complex)
    for i in range(N - 1, 0, -1):
        st.Renv[i - 1] = env_right(st.Renv[i], st.mps[i], st.W[i])
    return st


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
