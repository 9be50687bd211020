"""The 147-site chain (20 modes per electronic site, 16 levels) at D = 128 and D = 256.

At these sizes a whole oracle step takes minutes, so the CUDA path is checked on sampled
operations the oracle computes one by one (H_eff and the Lanczos exponential at one site, with
oracle-built environments) and on properties of the method that hold at any size: TDVP-PS
conserves the norm and the energy <H> exactly (each local step is a unitary exponential of a
Hermitian projected operator, the gauge shifts are exact), up to the Krylov tolerance in FP64 and
up to the TF32x3 contraction error in the mixed-precision sweep.  The Frenkel-Holstein
Hamiltonian (Eq. holstein) moves excitations between sites without creating any, so the total
excitation number sum_n <a_n^dag a_n> is a constant of the exact and of the continuous TDVP
motion; the split local steps keep it only up to the integrator's step error (each local
H_eff need not commute with the projected number operator), so it is checked at that level.
A random state is not in the one-exciton manifold: the sum is compared before and after, not
with 1.
"""
import numpy as np
import pytest

import workloads as wl
from workloads import PHASE_PER_CM_FS
from oracle import heff_apply, lanczos_expm, TDVPState, qr_rr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1907_12044_b300 as pkg  # noqa: E402
from gpu_util import (engine_for, debug_qr_or_rejected, oracle_centred, gauge_err, MIXED_TOL,  # noqa: E402
                      PREC_NAME, rel_err)


@pytest.fixture(scope="module")
def large128():
    p = wl.fmo_large()
    tens = wl.random_mps_tensors(p.phys_dims(), 128, seed=31)
    return p, tens


def _site_heff_and_expm_match_oracle(p, tens, site, D):
    """At `site`, with nothing taken from the CUDA path: the oracle right-canonicalises the seeded
    tensors, moves its own centre there by QR shifts and builds its own environments; the device
    does the same from the same tensors.  Compared: the device's gauge, H_eff x in FP64 and in
    every mixed mode, and the Lanczos exponential of the oracle's centre tensor."""
    mps, W, L, R = oracle_centred(p, tens, site)
    assert mps[site].shape[0] == D and mps[site].shape[2] == D
    eng = engine_for(p, tensors=tens)
    eng.move_center(0, site)
    g = gauge_err(eng.get_mps(0), mps, sorted({0, site - 1, site, site + 1, len(mps) - 1}))
    print(f"D = {D} site {site}: gauge {g:.1e}")
    assert g <= 1e-10
    rng = np.random.default_rng(site)
    x = rng.normal(size=mps[site].shape) + 1j * rng.normal(size=mps[site].shape)
    yo = heff_apply(L, W[site], R, x)
    y = eng.apply_heff(0, site, x)
    assert np.abs(y - yo).max() <= 1e-11 * np.abs(yo).max()
    for prec in pkg.MIXED_PRECISIONS:
        e = rel_err(eng.apply_heff(0, site, x, precision=prec), yo)
        print(f"D = {D} site {site}: {PREC_NAME[prec]} rel err {e:.2e}")
        assert e <= MIXED_TOL[prec], (prec, e)
    C = mps[site]
    tau = 10.0 * PHASE_PER_CM_FS / 2
    out, k = eng.debug_expm(0, site, -1j * tau, 1e-12, C)
    outo = lanczos_expm(lambda v: heff_apply(L, W[site], R, v), C, -1j * tau, 1e-12, 64)
    assert np.abs(out - outo).max() <= 1e-10 * np.abs(outo).max()
    eng.close()


def test_large_chain_heff_and_expm_match_oracle_at_d128(large128):
    p, tens = large128
    _site_heff_and_expm_match_oracle(p, tens, 5, 128)        # a 128 x 16 x 128 bath-mode site


def test_heff_and_expm_match_oracle_at_d256_with_the_largest_mpo_bond():
    """The site shapes of the D = 256 sweep, 256 x 16 x 256 with MPO bonds 9 x 9, on a 21-site
    chain with the large chain's bath modes (16 levels; 2 modes per electronic site), so that the
    oracle's own canonical form and environments take seconds rather than minutes."""
    p = wl.fmo_sized(n_modes=2, n_levels=16)
    tens = wl.random_mps_tensors(p.phys_dims(), 256, seed=34)
    assert TDVPState.start(p, D=1).W[10].shape[:2] == (9, 9)
    _site_heff_and_expm_match_oracle(p, tens, 10, 256)


# TF32x3 contractions carry about 1e-6 relative error per matvec at these magnitudes (the H_eff
# check above allows 2e-5 of max |y|).  The exponentials stay unitary to the Krylov tolerance,
# so the norm moves by little, but the energy of each local step is that of a perturbed H_eff:
# over the 2N - 1 = 293 local steps of a step, with ||H_eff|| about twice |<H>| for these random
# states (bath modes filled to ~7 quanta), the drift is bounded by 293 * 2 * 2e-6 ~ 1.2e-3 of |<H>|.
MIXED_ENERGY_REL = 2e-3
MIXED_NORM = 5e-5


def test_large_chain_step_at_d128_fp64_conserves_and_mixed_matches_fp64(large128):
    p, tens = large128
    a = engine_for(p, tensors=tens)
    b = engine_for(p, tensors=tens)
    P0, E0, n0 = a.observables(0)
    assert abs(n0 - 1.0) <= 1e-12
    a.step(10.0, precision=pkg.PREC_FP64)
    b.step(10.0, precision=pkg.PREC_TF32X3)
    Pa, Ea, na = a.observables(0)
    Pb, Eb, nb = b.observables(0)
    assert abs(na - 1.0) <= 1e-9
    assert abs(Ea - E0) <= 1e-9 * abs(E0)
    assert abs(Pa.sum() - P0.sum()) <= 1e-4 * P0.sum()
    # the mixed-precision step against the FP64 one: populations within 1e-4 (relative to the
    # largest), norm and energy within the bounds above
    assert np.abs(Pb - Pa).max() <= 1e-4 * np.abs(Pa).max()
    assert abs(nb - 1.0) <= MIXED_NORM
    assert abs(Eb - E0) <= MIXED_ENERGY_REL * abs(E0)
    a.close()
    b.close()


def test_large_chain_mixed_step_at_d256():
    p = wl.fmo_large()
    tens = wl.random_mps_tensors(p.phys_dims(), 256, seed=32)
    eng = engine_for(p, tensors=tens)
    assert max(int(t.shape[2]) for t in tens) == 256
    P0, E0, n0 = eng.observables(0)
    eng.step(10.0, precision=pkg.PREC_TF32X3, tol=1e-8)
    P1, E1, n1 = eng.observables(0)
    assert abs(n1 - 1.0) <= MIXED_NORM
    assert abs(E1 - E0) <= MIXED_ENERGY_REL * abs(E0)
    assert np.all(P1 >= -1e-6) and abs(P1.sum() - P0.sum()) <= 1e-4 * P0.sum()
    eng.close()


@pytest.fixture(scope="module")
def large256():
    p = wl.fmo_large()
    eng = engine_for(p, tensors=wl.random_mps_tensors(p.phys_dims(), 256, seed=33))
    yield eng
    eng.close()


@pytest.mark.parametrize("kernel", [0, -2, 4, 16])
def test_qr_at_bond_dim_256_matches_oracle(large256, kernel):
    """The gauge-shift QR at the largest bond dimension, in the shapes a D = 256 sweep meets:
    (Dl d) x Dr = 4096 x 256 in the chain, 512 x 256 and 256 x 256 at the square bonds near the
    ends (few columns per block, so the blocks of one realisation run close together), and a
    rank-64 matrix whose dropped rows go through the completion tail at n = 256."""
    eng = large256
    eng.set_option(pkg.OPT_QR_KERNEL, kernel)
    try:
        rng = np.random.default_rng(256 + kernel)
        cases = [rng.normal(size=(m, 256)) + 1j * rng.normal(size=(m, 256)) for m in (4096, 512, 256)]
        cases.append((rng.normal(size=(512, 64)) + 1j * rng.normal(size=(512, 64))) @ rng.normal(size=(64, 256)))
        for C in cases:
            out = debug_qr_or_rejected(eng, kernel, C)
            if out is None:
                continue
            Q, R = out
            Qo, Ro = qr_rr(C)
            n = C.shape[1]
            assert np.abs(Q.conj().T @ Q - np.eye(n)).max() < 1e-12
            assert np.abs(Q @ R - C).max() <= 1e-12 * np.abs(C).max()
            assert np.abs(Q - Qo).max() < 1e-10
            assert np.abs(R - Ro).max() < 1e-11 * np.abs(Ro).max()
    finally:
        eng.set_option(pkg.OPT_QR_KERNEL, -1)


def test_move_center_keeps_the_norm_at_d256(large256):
    eng = large256
    for site in (2, 70, 144, 0):
        eng.move_center(0, site)
        assert abs(eng.observables(0)[2] - 1.0) <= 1e-12
