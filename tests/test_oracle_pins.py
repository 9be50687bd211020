"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: a dense
Hamiltonian built term by term from Eq. holstein, a closed form, a library
routine on a case where it computes the same thing, an exact state-vector
propagation, the dense projector-splitting form of Eq. ps_trotter, or an
invariant of the method.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import (build_mpo, mpo_to_dense, qr_rr, lq_rr, expm_tridiag_e1, lanczos_expm,
                    product_mps, canonicalize_right, heff_apply, h0_apply, env_left, env_right,
                    mps_to_dense, TDVPState, tdvp_ps_step, populations, energy, norm,
                    mean_cumulative_deviation)
from oracle.dense import (hamiltonian_kron, product_state, propagate_exact, populations_dense,
                          projector_split_step)
from workloads import PHASE_PER_CM_FS, bond_dims


def _el_only(n, seed=5):
    rng = np.random.default_rng(seed)
    E = rng.uniform(12200, 12600, n)
    J = rng.normal(0, 40, (n, n))
    J = np.triu(J, 1)
    J = J + J.T
    order = list(rng.permutation(n))
    z = [np.zeros(0)] * n
    return wl.FHParams(E=E, J=J, omega=z, g=z, n_levels=[np.zeros(0, int)] * n, el_order=order,
                       energy_offset=float(E.mean()))


def _small_vibronic(levels=3, zpe=False):
    """3 electronic sites, 1-2 modes each: exercises left- and right-indexed MPO channels."""
    rng = np.random.default_rng(11)
    E = np.array([12400.0, 12450.0, 12300.0])
    J = np.array([[0, -60.0, 25.0], [-60.0, 0, 40.0], [25.0, 40.0, 0]])
    om = [np.array([150.0]), np.array([220.0, 480.0]), np.array([330.0])]
    g = [np.array([0.4]), np.array([0.3, 0.2]), np.array([0.5])]
    lev = [np.array([levels]), np.array([levels, 2]), np.array([levels])]
    return wl.FHParams(E=E, J=J, omega=om, g=g, n_levels=lev, el_order=[2, 0, 1],
                       energy_offset=12400.0, include_zpe=zpe)


# ---------------------------------------------------------------- MPO (Eq. mpo, Eq. holstein)

@pytest.mark.parametrize("maker", [wl.tiny_chain, lambda: _small_vibronic(),
                                   lambda: _small_vibronic(zpe=True), lambda: _el_only(7),
                                   lambda: _el_only(4), lambda: _el_only(5, seed=9),
                                   wl.two_level_rabi, wl.single_mode])
def test_mpo_equals_term_by_term_hamiltonian(maker):
    p = maker()
    H_mpo = mpo_to_dense(build_mpo(p))
    H_kron = hamiltonian_kron(p)
    assert H_mpo.shape == H_kron.shape
    assert np.abs(H_mpo - H_kron).max() <= 1e-12 * max(1.0, np.abs(H_kron).max())


def test_mpo_bond_dims_follow_min_rule():
    W = build_mpo(wl.tiny_chain())
    assert [w.shape[1] for w in W[:-1]] == [5, 5, 4, 3, 3]
    W = build_mpo(wl.fmo_sized())
    assert len(W) == 77
    assert max(w.shape[1] for w in W) == 9
    W7 = build_mpo(_el_only(7))
    assert [w.shape[1] for w in W7[:-1]] == [4, 6, 8, 8, 6, 4]


# ---------------------------------------------------------------- QR (Eq. QR) and LQ

def test_qr_full_rank_is_the_unique_positive_diagonal_qr():
    rng = np.random.default_rng(0)
    C = rng.normal(size=(40, 12)) + 1j * rng.normal(size=(40, 12))
    Q, R = qr_rr(C)
    Qn, Rn = np.linalg.qr(C)
    ph = np.diag(Rn) / np.abs(np.diag(Rn))
    Qn, Rn = Qn * ph, (Rn.T * ph.conj()).T
    assert np.allclose(Q, Qn, atol=1e-13) and np.allclose(R, Rn, atol=1e-12)
    assert np.allclose(np.tril(R, -1), 0)


def test_qr_rank_deficient_completion_rule():
    # rank 1: every later column is dropped and replaced by the first admissible e_p
    C = np.zeros((6, 3), dtype=complex)
    C[2, 0] = 2.0
    C[2, 1] = 1.0
    Q, R = qr_rr(C)
    assert np.allclose(Q.conj().T @ Q, np.eye(3), atol=1e-14)
    assert np.allclose(Q @ R, C, atol=1e-13)
    assert np.allclose(Q[:, 0], np.eye(6)[2]) and np.allclose(Q[:, 1], np.eye(6)[0])
    assert np.allclose(Q[:, 2], np.eye(6)[1])
    assert R[1, 1] == 0 and R[2, 2] == 0 and np.isclose(R[0, 1], 1.0)
    # generic rank-r matrix: orthonormal Q, C = QR within the drop tolerance
    rng = np.random.default_rng(1)
    X = (rng.normal(size=(30, 4)) + 1j * rng.normal(size=(30, 4))) @ (rng.normal(size=(4, 9)))
    Q, R = qr_rr(X)
    assert np.allclose(Q.conj().T @ Q, np.eye(9), atol=1e-13)
    assert np.abs(Q @ R - X).max() < 1e-11
    assert np.sum(np.abs(np.diag(R)) > 0) == 4


def test_qr_at_bond_dimension_256():
    """The sizes of a D = 256 sweep: full rank against the phase-normalised library QR, and a
    rank-64 matrix whose dropped columns are completed (orthonormal Q, C = QR, 64 kept)."""
    rng = np.random.default_rng(256)
    C = rng.normal(size=(512, 256)) + 1j * rng.normal(size=(512, 256))
    Q, R = qr_rr(C)
    Qn, Rn = np.linalg.qr(C)
    ph = np.diag(Rn) / np.abs(np.diag(Rn))
    Qn, Rn = Qn * ph, (Rn.T * ph.conj()).T
    assert np.abs(Q - Qn).max() < 1e-12 and np.abs(R - Rn).max() < 1e-11 * np.abs(Rn).max()
    X = (rng.normal(size=(512, 64)) + 1j * rng.normal(size=(512, 64))) @ rng.normal(size=(64, 256))
    Q, R = qr_rr(X)
    assert np.abs(Q.conj().T @ Q - np.eye(256)).max() < 1e-12
    assert np.abs(Q @ R - X).max() < 1e-12 * np.abs(X).max()
    assert np.sum(np.abs(np.diag(R)) > 0) == 64


def test_lq_orthonormal_rows():
    rng = np.random.default_rng(2)
    C = rng.normal(size=(8, 30)) + 1j * rng.normal(size=(8, 30))
    Dm, Qr = lq_rr(C)
    assert np.allclose(Qr @ Qr.conj().T, np.eye(8), atol=1e-13)
    assert np.allclose(Dm @ Qr, C, atol=1e-12)
    assert np.allclose(np.triu(Dm, 1), 0)


# ---------------------------------------------------------------- Krylov exponential

def test_expm_tridiag_matches_dense_expm():
    rng = np.random.default_rng(3)
    for k in (1, 2, 5, 17, 40):
        a = rng.normal(size=k) * 3
        b = np.abs(rng.normal(size=k - 1)) + 0.1
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        z = -0.7j
        ref = sla.expm(z * T)[:, 0]
        assert np.allclose(expm_tridiag_e1(a, b, z), ref, atol=1e-13)


def test_tridiagonal_exponential_at_wide_exponents():
    """exp(-i theta T) e_1 for theta ||T|| from 30 to 6000 against the Pade scaling-and-squaring
    matrix exponential (a different method from the oracle's eigendecomposition), in the regime
    where a Chebyshev series needs hundreds of terms or substeps; unitary."""
    rng = np.random.default_rng(7)
    k = 32
    a = rng.normal(size=k) * 100
    b = np.abs(rng.normal(size=k - 1)) * 50 + 1
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    lam = np.linalg.eigvalsh(T)
    for x in (30.0, 250.0, 1500.0, 6000.0):
        theta = x / (0.5 * (lam[-1] - lam[0]))
        ref = sla.expm(-1j * theta * T)[:, 0]
        out = expm_tridiag_e1(a, b, -1j * theta)
        assert np.abs(out - ref).max() < 1e-10
        assert abs(np.linalg.norm(out) - 1.0) < 1e-12


def test_lanczos_matches_dense_expm_and_converges():
    rng = np.random.default_rng(4)
    n = 80
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    H = (X + X.conj().T) / 2
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    ref = sla.expm(-0.3j * H) @ v
    errs = []
    for tol in (1e-4, 1e-8, 1e-12):
        ks = []
        out = lanczos_expm(lambda x: H @ x, v, -0.3j, tol=tol, kmax=80, stats=ks)
        errs.append(np.linalg.norm(out - ref))
        assert errs[-1] < 50 * tol
    assert errs[0] > errs[1] > errs[2]
    # full dimension: exact whatever the tolerance
    out = lanczos_expm(lambda x: H[:6, :6] @ x, v[:6], -5.0j, tol=0.0, kmax=60)
    assert np.allclose(out, sla.expm(-5.0j * H[:6, :6]) @ v[:6], atol=1e-12)
    # norm is conserved (unitary integrator, Sec. II.A.2 TDVP-PS)
    assert abs(np.linalg.norm(ref) - np.linalg.norm(v)) < 1e-10


# ---------------------------------------------------------------- MPS, environments, H_eff

def test_product_mps_is_right_canonical_product_state():
    p = wl.tiny_chain()
    d = p.phys_dims()
    for D in (1, 4, 16, 32):
        mps = product_mps(d, bond_dims(d, D), p.occupied())
        for A in mps[1:]:
            Dl = A.shape[0]
            M = A.reshape(Dl, -1)
            assert np.allclose(M @ M.conj().T, np.eye(Dl))
        assert np.allclose(mps_to_dense(mps), product_state(p))


def test_right_canonicalisation_keeps_the_state_and_survives_any_scale():
    """canonicalize_right (Eq. QR, right-to-left): sites 1..N-1 right-canonical (Eq. rcanon), the
    dense state equal to the raw tensors' product divided by its norm (no phase: every LQ factor
    has a positive diagonal), and tensors scaled by 1e70 each (a product of 1e420, beyond the
    float64 range, on this 6-site chain) give the same tensors."""
    p = wl.tiny_chain()
    d = p.phys_dims()
    assert len(d) == 6
    tens = wl.random_mps_tensors(d, 6, seed=15)
    psi = mps_to_dense(tens)
    psi = psi / np.linalg.norm(psi)
    mps = canonicalize_right(tens)
    for A in mps[1:]:
        M = A.reshape(A.shape[0], -1)
        assert np.allclose(M @ M.conj().T, np.eye(A.shape[0]), atol=1e-13)
    assert np.allclose(mps_to_dense(mps), psi, atol=1e-12)
    big = canonicalize_right([1e70 * t for t in tens])
    for A, B in zip(mps, big):
        assert np.all(np.isfinite(B)) and np.allclose(A, B, atol=1e-12)


def _dense_heff(p, mps, i):
    """P^H H P for the site projector of site i, from the dense H (no environments)."""
    H = hamiltonian_kron(p)
    d = p.phys_dims()
    UL = np.ones((1, 1))
    for A in mps[:i]:
        UL = np.einsum("xa,asb->xsb", UL, A).reshape(-1, A.shape[2])
    UR = np.ones((1, 1))
    for A in mps[:i:-1]:
        UR = np.einsum("asb,bx->asx", A, UR).reshape(A.shape[0], -1)
    P = np.kron(np.kron(UL, np.eye(d[i])), UR.T)
    return P.conj().T @ H @ P


def test_heff_env_and_h0_match_dense_projection():
    p = _small_vibronic()
    W = build_mpo(p)
    d = p.phys_dims()
    tens = wl.random_mps_tensors(d, 4, seed=8)
    # left-canonical sites < i, right-canonical sites > i, random centre
    i = 3
    mps = canonicalize_right(tens)
    for j in range(i):
        Dl, dj, Dr = mps[j].shape
        Q, Rm = qr_rr(mps[j].reshape(Dl * dj, Dr))
        mps[j] = Q.reshape(Dl, dj, Dr)
        mps[j + 1] = np.einsum("ab,bsc->asc", Rm, mps[j + 1])
    L = np.ones((1, 1, 1), complex)
    for j in range(i):
        L = env_left(L, mps[j], W[j])
    R = np.ones((1, 1, 1), complex)
    for j in range(len(d) - 1, i, -1):
        R = env_right(R, mps[j], W[j])
    Hd = _dense_heff(p, mps, i)
    x = np.random.default_rng(9).normal(size=mps[i].shape) + 0j
    assert np.allclose(heff_apply(L, W[i], R, x).reshape(-1), Hd @ x.reshape(-1), atol=1e-10)
    assert np.allclose(Hd, Hd.conj().T, atol=1e-10)
    # zero-site: bond between i and i+1 after the QR of site i
    Dl, di, Dr = mps[i].shape
    Q, Rm = qr_rr(mps[i].reshape(Dl * di, Dr))
    mps[i] = Q.reshape(Dl, di, Dr)
    L2 = env_left(L, mps[i], W[i])
    H = hamiltonian_kron(p)
    UL = np.ones((1, 1))
    for A in mps[: i + 1]:
        UL = np.einsum("xa,asb->xsb", UL, A).reshape(-1, A.shape[2])
    UR = np.ones((1, 1))
    for A in mps[:i:-1]:
        UR = np.einsum("asb,bx->asx", A, UR).reshape(A.shape[0], -1)
    P = np.kron(UL, UR.T)
    H0 = P.conj().T @ H @ P
    y = np.random.default_rng(10).normal(size=Rm.shape) + 1j
    assert np.allclose(h0_apply(L2, R, y).reshape(-1), H0 @ y.reshape(-1), atol=1e-10)


# ---------------------------------------------------------------- closed forms

def test_rabi_oscillation_closed_form():
    p = wl.two_level_rabi()
    st = TDVPState.start(p, D=2)
    Delta = (p.E[0] - p.E[1])
    J = p.J[0, 1]
    Om = np.sqrt(Delta ** 2 + 4 * J ** 2)
    for s in range(1, 31):
        tdvp_ps_step(st, 10.0)
        t = 10.0 * s * PHASE_PER_CM_FS
        P1 = 1 - 4 * J ** 2 / Om ** 2 * np.sin(Om * t / 2) ** 2
        assert abs(populations(st, p)[0] - P1) < 1e-11


def test_displaced_oscillator_phonon_number():
    # exciton fixed on one site: <b+b>(t) = 2 g^2 (1 - cos w t) for an untruncated mode
    p = wl.single_mode(omega=200.0, S=0.1, levels=14)
    st = TDVPState.start(p, D=14)
    H = hamiltonian_kron(p)
    psi0 = product_state(p)
    nb = np.kron(np.eye(2), np.diag(np.arange(14.0)))
    for s in range(1, 21):
        tdvp_ps_step(st, 10.0)
        psi = mps_to_dense(st.mps)
        t = 10.0 * s
        exact = propagate_exact(H, psi0, [t])[0]
        assert np.allclose(psi, exact, atol=1e-10)
        closed = 2 * 0.1 * (1 - np.cos(200.0 * PHASE_PER_CM_FS * t))
        assert abs(np.vdot(psi, nb @ psi).real - closed) < 1e-7


def test_no_coupling_keeps_populations():
    p = wl.tiny_chain()
    p.J = np.zeros_like(p.J)
    st = TDVPState.start(p, D=8)
    for _ in range(5):
        tdvp_ps_step(st, 10.0)
    assert np.allclose(populations(st, p), [1.0, 0.0], atol=1e-12)


# ---------------------------------------------------------------- exactness and invariants

@pytest.mark.slow
def test_full_bond_dim_is_exact_over_100_steps():
    """At maximal bond dims every projector is the identity and TDVP-PS is exact."""
    p = wl.tiny_chain()
    assert max(bond_dims(p.phys_dims(), 10 ** 6)) == 32
    st = TDVPState.start(p, D=32)
    H = hamiltonian_kron(p)
    psi0 = product_state(p)
    times = 10.0 * np.arange(1, 101)
    exact = propagate_exact(H, psi0, times)
    worst = 0.0
    for s in range(100):
        tdvp_ps_step(st, 10.0)
        worst = max(worst, np.abs(populations(st, p) - populations_dense(exact[s], p)).max())
    assert worst <= 1e-10


def test_truncated_matches_dense_projector_splitting():
    """At truncated D the oracle equals Eq. ps_trotter with dense exponentials."""
    p = _small_vibronic(levels=2)
    H = hamiltonian_kron(p)
    for start in ("product", "random"):
        if start == "product":
            st = TDVPState.start(p, D=3)
        else:
            st = TDVPState.start(p, tensors=wl.random_mps_tensors(p.phys_dims(), 3, seed=4))
        psi = mps_to_dense(st.mps)
        mps = [a.copy() for a in st.mps]
        for _ in range(4):
            tdvp_ps_step(st, 10.0)
            psi, mps = projector_split_step(psi, p, mps, H, 10.0)
            assert np.abs(mps_to_dense(st.mps) - psi).max() < 1e-11
            assert np.abs(populations(st, p) - populations_dense(psi, p)).max() < 1e-11


def test_norm_energy_and_population_sum_are_conserved():
    p = wl.tiny_chain()
    st = TDVPState.start(p, tensors=wl.random_mps_tensors(p.phys_dims(), 8, seed=12))
    E0 = energy(st)
    for _ in range(8):
        tdvp_ps_step(st, 10.0)
        assert abs(norm(st) - 1) < 1e-11
        assert abs(energy(st) - E0) < 1e-9 * max(1, abs(E0))
        # population of a random state need not sum to 1, but it is conserved
    p2 = wl.tiny_chain()
    st2 = TDVPState.start(p2, D=8)
    for _ in range(8):
        tdvp_ps_step(st2, 10.0)
        assert abs(populations(st2, p2).sum() - 1) < 1e-12


def test_second_order_in_dt():
    """Global error of the symmetric split is O(tau^2) at fixed D (Eq. ps_trotter)."""
    p = wl.tiny_chain()
    tens = wl.random_mps_tensors(p.phys_dims(), 8, seed=3)

    def run(dt, T=80.0):
        st = TDVPState.start(p, tensors=tens)
        for _ in range(int(round(T / dt))):
            tdvp_ps_step(st, dt)
        return mps_to_dense(st.mps)

    ref = run(1.25)
    e = [np.linalg.norm(run(dt) - ref) for dt in (20.0, 10.0, 5.0)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0


def test_mean_cumulative_deviation_closed_form():
    t = np.linspace(0, 100, 201)
    P = np.stack([0.5 + 0.01 * t / 100, 0.5 - 0.01 * t / 100], axis=1)
    Pref = np.full_like(P, 0.5)
    # sum_n |dP| = 0.02 t/100, integral = 0.01 t^2/100, divided by 2 t
    assert abs(mean_cumulative_deviation(t, P, Pref) - 0.01 * 100 / 100 / 2) < 1e-12


# ---------------------------------------------------------------- observables against the dense state

def _dense_observable_deviation(p, D, seed, norm_fn=None, energy_fn=None, pops_fn=None,
                                mpo_fn=None):
    """Largest relative deviation of the oracle's norm, energy and populations from the dense
    state vector of the same (random, non-canonical, unnormalised) MPS: ||psi||,
    <psi|H|psi>/<psi|psi> with the Kronecker-built H, and <psi|n_m|psi>/<psi|psi>.  The keyword
    arguments replace an oracle function (planted-mistake tests)."""
    import types
    norm_fn, energy_fn = norm_fn or norm, energy_fn or energy
    pops_fn, mpo_fn = pops_fn or populations, mpo_fn or build_mpo
    tens = [2.0 * t for t in wl.random_mps_tensors(p.phys_dims(), D, seed=seed)]
    st = types.SimpleNamespace(mps=tens, W=mpo_fn(p))
    psi = mps_to_dense(tens)
    H = hamiltonian_kron(p)
    n_d = np.linalg.norm(psi)
    E_d = np.vdot(psi, H @ psi).real / n_d ** 2
    P_d = populations_dense(psi, p)
    assert abs(n_d - 1) > 0.1                      # a norm that is always 1 cannot pass
    return max(abs(norm_fn(st) - n_d) / n_d, abs(energy_fn(st) - E_d) / max(1.0, abs(E_d)),
               np.abs(pops_fn(st, p) - P_d).max())


@pytest.mark.parametrize("maker,D,seed", [(wl.tiny_chain, 8, 21), (wl.tiny_chain, 32, 22),
                                          (lambda: _small_vibronic(), 3, 23),
                                          (lambda: _small_vibronic(zpe=True), 4, 24)])
def test_norm_energy_populations_match_dense_state(maker, D, seed):
    """norm() = ||psi||, energy() = <psi|H|psi>/<psi|psi> and populations() of Eq. error on
    random truncated states, against the dense vector and the term-by-term H of Eq. holstein."""
    assert _dense_observable_deviation(maker(), D, seed) < 1e-12


# ---------------------------------------------------------------- product start against exact dynamics

@pytest.mark.slow
def test_product_start_completion_tracks_exact_dynamics():
    """The completion rows of the product start (reading of Sec. II.C) span the directions H
    reaches from the product state: at D = 16 the truncated TDVP-PS follows the exact
    state-vector populations over 400 fs.  The s-first order freezes them (error 0.53)."""
    p = wl.tiny_chain()
    st = TDVPState.start(p, D=16)
    exact = propagate_exact(hamiltonian_kron(p), product_state(p), 10.0 * np.arange(1, 41))
    worst = 0.0
    for s in range(40):
        tdvp_ps_step(st, 10.0)
        worst = max(worst, np.abs(populations(st, p) - populations_dense(exact[s], p)).max())
    assert worst < 2e-5
    assert np.abs(populations(st, p) - [1.0, 0.0]).max() > 0.1       # population did move
