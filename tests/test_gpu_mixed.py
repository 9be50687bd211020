"""Mixed-precision (tensor-core) contractions against the FP64 oracle.

Each mode rounds the operands of the real products to its input format: TF32 keeps 11
significant bits (unit roundoff u = 2^-11), BF16 8 (u = 2^-8); the compensated x3 modes carry
the rounded remainder as a second term, so their products are good to about u^2 of the format
(limited to ~FP32 by the accumulator for TF32x3, ~2^-16 for BF16x3); the 3M (Gauss) form adds
one more rounding (of re + im) per operand and a subtraction of larger partial products.  A
complex contraction of many terms then carries a relative error of a few u of its terms.  The
bounds (tests/gpu_util.py) are 10 u (4M), 20 u (3M), with the x3 modes at 2e-5 (TF32x3) and
10 x 2^-16 (BF16x3): ||y - y_ref|| / ||y_ref|| against the oracle's complex128 contraction.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import heff_apply, h0_apply, TDVPState, tdvp_ps_step, populations

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1907_12044_b300 as pkg  # noqa: E402
from gpu_util import (engine_for, oracle_centred, gauge_err, rel_pop_err, MIXED_TOL as TOL,  # noqa: E402
                      PREC_NAME as NAME, rel_err as _rel)


@pytest.fixture
def c1_random():
    """A fresh engine per test: moving the centre out and back re-gauges the sites it passes
    (the LQ of R_0 B_1 is not R_0 B_1 itself), so only a context that has made exactly the
    oracle's gauge shifts holds the oracle's gauge."""
    p = wl.fmo_sized()
    tens = wl.random_mps_tensors(p.phys_dims(), 64, seed=21)
    eng = engine_for(p, tensors=tens)
    yield p, eng, tens
    eng.close()


@pytest.mark.parametrize("site", [0, 1, 5, 38, 76])
def test_mixed_heff_matches_oracle(c1_random, site):
    """H_eff x in every mixed mode against the oracle's contraction over its own gauge and
    environments (built from the seeded tensors alone)."""
    p, eng, tens = c1_random
    mps, W, L, R = oracle_centred(p, tens, site)
    eng.move_center(0, site)
    assert gauge_err(eng.get_mps(0), mps, sorted({0, site, len(mps) - 1})) <= 1e-10
    rng = np.random.default_rng(100 + site)
    x = rng.normal(size=mps[site].shape) + 1j * rng.normal(size=mps[site].shape)
    yo = heff_apply(L, W[site], R, x)
    errs = {prec: _rel(eng.apply_heff(0, site, x, precision=prec), yo) for prec in pkg.MIXED_PRECISIONS}
    print(f"site {site}: rel err " + "  ".join(f"{NAME[q]} {e:.2e}" for q, e in errs.items()))
    for prec, e in errs.items():
        assert e <= TOL[prec], (prec, e)


@pytest.mark.parametrize("bond", [0, 4, 40, 75])
def test_mixed_zero_site_matches_oracle(c1_random, bond):
    """H0 on the bond (bond, bond + 1): the oracle's left environment through site `bond` (centre
    moved to bond + 1) and right environment of the sites after `bond` (centre at bond)."""
    p, eng, tens = c1_random
    _, _, _, R = oracle_centred(p, tens, bond)
    mps1, W, L, _ = oracle_centred(p, tens, bond + 1)
    eng.move_center(0, bond + 1)
    assert gauge_err(eng.get_mps(0), mps1, sorted({0, bond, bond + 1})) <= 1e-10
    Db = mps1[bond].shape[2]
    rng = np.random.default_rng(7 + bond)
    x = rng.normal(size=(Db, Db)) + 1j * rng.normal(size=(Db, Db))
    yo = h0_apply(L, R, x)
    assert _rel(eng.apply_h0(0, bond, x, precision=pkg.PREC_FP64), yo) <= 1e-11
    for prec in pkg.MIXED_PRECISIONS:
        e = _rel(eng.apply_h0(0, bond, x, precision=prec), yo)
        print(f"bond {bond}: {NAME[prec]} rel err {e:.2e}")
        assert e <= TOL[prec], (prec, e)


# relative population error over 10 steps: the matvec bound above times a few (the error of
# each local exponential adds up over the 2N - 1 site updates of a step and over the steps)
STEP_TOL = {pkg.PREC_TF32X3: 1e-5, pkg.PREC_TF32: 3e-3, pkg.PREC_BF16X3: 3e-4, pkg.PREC_BF16: 2.5e-2,
            pkg.PREC_TF32_3M: 6e-3, pkg.PREC_BF16_3M: 5e-2}


@pytest.mark.parametrize("prec", list(STEP_TOL))
def test_mixed_steps_track_fp64_oracle(prec):
    tol = STEP_TOL[prec]
    p = wl.tiny_chain()
    tens = wl.random_mps_tensors(p.phys_dims(), 16, seed=9)
    eng = engine_for(p, tensors=tens)
    st = TDVPState.start(p, tensors=tens)
    worst = 0.0
    for _ in range(10):
        eng.step(10.0, precision=prec, tol=1e-10)
        tdvp_ps_step(st, 10.0)
        worst = max(worst, rel_pop_err(eng.observables(0)[0], populations(st, p)))
    print(f"tiny chain, precision {prec}: worst relative population error {worst:.2e}")
    assert worst <= tol


def test_mixed_fmo_step_tracks_fp64_oracle():
    p = wl.fmo_sized()
    eng = engine_for(p, D=64)
    st = TDVPState.start(p, D=64)
    eng.step(10.0, precision=pkg.PREC_TF32X3, tol=1e-10)
    tdvp_ps_step(st, 10.0)
    err = rel_pop_err(eng.observables(0)[0], populations(st, p))
    print(f"FMO-sized chain, one TF32x3 step: relative population error {err:.2e}")
    assert err <= 1e-5


def test_mixed_matvecs_with_fp64_environments_track_the_oracle():
    """TDVP_OPT_ENV_FP64: the mixed sweep with the environment updates kept in FP64 (only the
    Lanczos matvecs on the tensor cores) stays on the FP64 oracle like the all-tensor-core sweep."""
    p = wl.tiny_chain()
    tens = wl.random_mps_tensors(p.phys_dims(), 16, seed=9)
    eng = engine_for(p, tensors=tens)
    eng.set_option(pkg.OPT_ENV_FP64, 1)
    st = TDVPState.start(p, tensors=tens)
    worst = 0.0
    for _ in range(10):
        eng.step(10.0, precision=pkg.PREC_TF32X3, tol=1e-10)
        tdvp_ps_step(st, 10.0)
        worst = max(worst, rel_pop_err(eng.observables(0)[0], populations(st, p)))
    print(f"tiny chain, TF32x3 with FP64 environments: worst relative population error {worst:.2e}")
    assert worst <= STEP_TOL[pkg.PREC_TF32X3]
    eng.close()
