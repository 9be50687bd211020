"""Two-site TDVP-PS with SVD truncation (the adaptive-bond variant mentioned at the end of
Sec. II.A.2, TDVP-PS paragraph).

TEST INFRASTRUCTURE (oracle); see the package docstring.

The paper names the two-site form only as the way to grow the bond dimension from a weakly
correlated start; the steps below are the two-site analogue of its one-site split
(Eq. ps_trotter, Eq. tdvp2_C, Eq. tdvp2_D), with the pair of sites in place of the site and
the site in place of the bond:

* left to right with tau/2, for the pairs (i, i+1), i = 1..N-1: the pair tensor
  Theta = A_i A_{i+1} is evolved forward with the two-site effective Hamiltonian (the
  environments of Eq. tdvp1_h1i / tdvp1_hiN around two MPO tensors), split by a truncated
  SVD (Eq. SVD: site i <- U, left-canonical; site i+1 <- Lambda V^dag), the left environment
  of site i+1 is updated, and unless i+1 is the last site, site i+1 is evolved backward with
  +i tau/2 under the one-site H[i+1] (Eq. tdvp2_C with the opposite sign);
* the mirror sweep right to left with tau/2, for the pairs (i-1, i), i = N..2, with the
  split site i <- V^dag (right-canonical), site i-1 <- U Lambda, and the backward one-site
  step of site i-1 unless it is the first site.

Readings:
* the turning pair (N-1, N) is evolved by tau/2 at the end of the first sweep and again at the
  start of the second, with the split in between (no merge into one exponential: the split is
  where the bond may grow);
* the truncation keeps at most D singular values and only those above zeta * ||Lambda||
  (criteria i and ii of Eq. SVD) and never fewer than one; singular values at or below 1e-14
  of the largest are dropped with the rest; the kept weight is not renormalised (the norm
  falls by the discarded weight, as in the paper's compression);
* the Krylov exponential and its stopping rule are those of the one-site oracle.
"""
from __future__ import annotations

import numpy as np

from workloads import PHASE_PER_CM_FS
from .linalg import lanczos_expm
from .mps import heff_apply, env_left, env_right

SV_FLOOR = 1e-14
_PATH = ("greedy", 1e15)


def heff2_apply(L, W1, W2, R, T):
    """Two-site effective Hamiltonian: out[x,t,u,y] =
    sum L[x,w,a] W1[w,v,t,s] W2[v,q,u,r] T[a,s,r,b] R[y,q,b]."""
    return np.einsum("xwa,wvts,vqur,asrb,yqb->xtuy", L, W1, W2, T, R, optimize=_PATH)


def truncated_svd(M, D, zeta=0.0):
    """M = U diag(S) Vh truncated to at most D values above zeta*||S|| (at least one)."""
    U, S, Vh = np.linalg.svd(M, full_matrices=False)
    nrm = np.linalg.norm(S)
    keep = int(np.sum(S > max(zeta * nrm, SV_FLOOR * S[0]))) if S[0] > 0 else 0
    keep = max(1, min(D, keep))
    return U[:, :keep], S[:keep], Vh[:keep]


def tdvp2_step(W, mps, dt_fs, D, zeta=0.0, tol=1e-12, kmax=60):
    """One two-site TDVP-PS step of dt on an MPS with its centre at site 0 (sites 1..N-1
    right-canonical), for the MPO W.  Returns the new tensors, centre again at site 0."""
    tau = dt_fs * PHASE_PER_CM_FS
    A = [np.array(t, dtype=complex) for t in mps]
    N = len(A)
    one = np.ones((1, 1, 1), dtype=complex)
    L = [None] * N
    R = [None] * N
    L[0] = one
    R[N - 1] = one
    for i in range(N - 1, 0, -1):
        R[i - 1] = env_right(R[i], A[i], W[i])

    def evolve_pair(i, t):
        Dl, d1, _ = A[i].shape
        _, d2, Dr = A[i + 1].shape
        T = np.einsum("asb,bur->asur", A[i], A[i + 1])
        T = lanczos_expm(lambda x: heff2_apply(L[i], W[i], W[i + 1], R[i + 1], x), T, -1j * t, tol, kmax)
        return T.reshape(Dl * d1, d2 * Dr), (Dl, d1, d2, Dr)

    for i in range(N - 1):
        M, (Dl, d1, d2, Dr) = evolve_pair(i, tau / 2)
        U, S, Vh = truncated_svd(M, D, zeta)
        A[i] = U.reshape(Dl, d1, -1)
        A[i + 1] = (S[:, None] * Vh).reshape(-1, d2, Dr)
        L[i + 1] = env_left(L[i], A[i], W[i])
        if i + 1 < N - 1:
            A[i + 1] = lanczos_expm(lambda x: heff_apply(L[i + 1], W[i + 1], R[i + 1], x), A[i + 1],
                                    1j * tau / 2, tol, kmax)
    for i in range(N - 1, 0, -1):
        M, (Dl, d1, d2, Dr) = evolve_pair(i - 1, tau / 2)
        U, S, Vh = truncated_svd(M, D, zeta)
        A[i] = Vh.reshape(-1, d2, Dr)
        A[i - 1] = (U * S).reshape(Dl, d1, -1)
        R[i - 1] = env_right(R[i], A[i], W[i])
        if i - 1 > 0:
            A[i - 1] = lanczos_expm(lambda x: heff_apply(L[i - 1], W[i - 1], R[i - 1], x), A[i - 1],
                                    1j * tau / 2, tol, kmax)
    return A
