"""Gauge-shift decomposition and Krylov exponential for the oracle.

TEST INFRASTRUCTURE (oracle); see the package docstring.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh_tridiagonal

# Columns whose residual after two Gram-Schmidt passes is below this fraction of
# ||C||_F count as linearly dependent (reading of the QR in Eq. QR for
# rank-deficient C, see qr_rr).
RANK_RTOL = 1e-13


def qr_rr(C, rtol=RANK_RTOL):
    """C = Q R with Q (m x n) orthonormal columns, R (n x n) upper triangular (Eq. QR).

    Column-by-column classical Gram-Schmidt with one re-orthogonalisation pass
    ("twice is enough").  For full-rank C this is the unique QR with a positive
    real diagonal.  Reading for rank-deficient C (the paper's weakly correlated
    start, Sec. II.C): a column whose residual norm is <= rtol*||C||_F is dropped
    (R[j,j] = 0) and Q[:, j] is completed from the first standard basis vector
    e_p (p ascending over the row index) whose distance to span(Q[:, :j]) is at
    least 1/2, i.e. 1 - ||Q[p, :j]||^2 >= 1/4; if none qualifies, the p with the
    largest such distance (first on ties).  e_p is orthogonalised with the same
    two passes and normalised.
    """
    C = np.asarray(C, dtype=complex)
    m, n = C.shape
    assert m >= n, "qr_rr expects a tall or square matrix"
    Q = np.zeros((m, n), dtype=complex)
    R = np.zeros((n, n), dtype=complex)
    thresh = rtol * np.linalg.norm(C)
    for j in range(n):
        c = C[:, j].copy()
        for _ in range(2):
            h = Q[:, :j].conj().T @ c
            c = c - Q[:, :j] @ h
            R[:j, j] += h
        nr = np.linalg.norm(c)
        if nr > thresh:
            Q[:, j] = c / nr
            R[j, j] = nr
            continue
        dist2 = 1.0 - np.sum(np.abs(Q[:, :j]) ** 2, axis=1)
        ok = np.nonzero(dist2 >= 0.25)[0]
        p = int(ok[0]) if ok.size else int(np.argmax(dist2))
        e = np.zeros(m, dtype=complex)
        e[p] = 1.0
        for _ in range(2):
            e = e - Q[:, :j] @ (Q[:, :j].conj().T @ e)
        Q[:, j] = e / np.linalg.norm(e)
    return Q, R


def lq_rr(C, rtol=RANK_RTOL):
    """C = Dm Qr with Qr (m x n, m <= n) orthonormal rows: QR of the transpose.

    This is the right-to-left gauge shift ("RQ" in Sec. II.A): C^T = Q R gives
    C = R^T Q^T, and the rows of Q^T are orthonormal.
    """
    Q, R = qr_rr(np.asarray(C).T, rtol)
    return R.T, Q.T


def expm_tridiag_e1(alpha, beta, z):
    """exp(z T) e_1 for the real symmetric tridiagonal T = tridiag(beta, alpha, beta).

    T = U diag(lam) U^T, so exp(zT) e_1 = U (exp(z lam) * U[0, :]).
    """
    alpha = np.asarray(alpha, float)
    k = alpha.size
    if k == 1:
        return np.array([np.exp(z * alpha[0])])
    lam, U = eigh_tridiagonal(alpha, np.asarray(beta, float)[: k - 1])
    return U @ (np.exp(z * lam) * U[0, :])


def lanczos_expm(matvec, v, z, tol=1e-12, kmax=60, dim=None, stats=None):
    """exp(z H) v for Hermitian H given by ``matvec`` and z = -i*tau (Sec. II.A.2, TDVP-PS).

    Lanczos with full re-orthogonalisation (two classical Gram-Schmidt passes
    against every earlier Krylov vector) builds V_k and T_k; the result is
    ||v|| V_k exp(z T_k) e_1.  The Krylov dimension grows until the a-posteriori
    estimate ||v|| beta_k |[exp(z T_k) e_1]_k| is <= tol, or k reaches kmax or the
    dimension of the space (the paper stops the iteration once the evolved state has
    converged, Sec. II.A.2; this estimate is the reading of that test).
    """
    shape = v.shape
    v = np.asarray(v, dtype=complex).reshape(-1)
    nv = np.linalg.norm(v)
    n = v.size if dim is None else dim
    kcap = min(kmax, n)
    if nv == 0.0:
        return v.reshape(shape).copy()
    V = [v / nv]
    alpha, beta = [], []
    c = None
    for j in range(kcap):
        w = np.asarray(matvec(V[j].reshape(shape)), dtype=complex).reshape(-1)
        Vm = np.array(V)
        h1 = Vm.conj() @ w
        w = w - Vm.T @ h1
        h2 = Vm.conj() @ w
        w = w - Vm.T @ h2
        alpha.append(float(np.real(h1[j] + h2[j])))
        b = float(np.linalg.norm(w))
        c = expm_tridiag_e1(alpha, beta, z)
        err = nv * b * abs(c[-1])
        if err <= tol or j + 1 == kcap:
            break
        beta.append(b)
        V.append(w / b)
    if stats is not None:
        stats.append(len(alpha))
    out = nv * (np.array(V).T @ c)
    return out.reshape(shape)
