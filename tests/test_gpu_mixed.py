"""Mixed-precision (tensor-core) Lanczos matvecs against the FP64 oracle.

TF32 rounds every operand to 11 significant bits (relative error <= 2^-12 per operand), so a
complex contraction carries a relative error of order 1e-3 of its terms; the compensated mode
(hi/lo split, three products) reaches FP32-level products (~1e-6).  The bounds below are those
orders with a margin: ||y - y_ref|| / ||y_ref|| <= 5e-3 (TF32) and <= 2e-5 (TF32x3).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import heff_apply, h0_apply, env_left, env_right, TDVPState, tdvp_ps_step, populations

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1907_12044_b300 as pkg  # noqa: E402
from gpu_util import engine_for, rel_pop_err  # noqa: E402

TOL = {pkg.PREC_TF32: 5e-3, pkg.PREC_TF32X3: 2e-5}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def c1_random():
    p = wl.fmo_sized()
    tens = wl.random_mps_tensors(p.phys_dims(), 64, seed=21)
    return p, engine_for(p, tensors=tens)


@pytest.mark.parametrize("site", [0, 1, 5, 38, 76])
def test_mixed_heff_matches_oracle(c1_random, site):
    p, eng = c1_random
    W = TDVPState.start(p, D=1).W
    eng.move_center(0, site)
    try:
        mps = eng.get_mps(0)
        L = np.ones((1, 1, 1), complex)
        for j in range(site):
            L = env_left(L, mps[j], W[j])
        R = np.ones((1, 1, 1), complex)
        for j in range(len(mps) - 1, site, -1):
            R = env_right(R, mps[j], W[j])
        rng = np.random.default_rng(100 + site)
        x = rng.normal(size=mps[site].shape) + 1j * rng.normal(size=mps[site].shape)
        yo = heff_apply(L, W[site], R, x)
        errs = {}
        for prec in (pkg.PREC_TF32, pkg.PREC_TF32X3):
            y = eng.apply_heff(0, site, x, precision=prec)
            errs[prec] = _rel(y, yo)
        print(f"site {site}: rel err TF32 {errs[pkg.PREC_TF32]:.2e}  TF32x3 {errs[pkg.PREC_TF32X3]:.2e}")
        for prec, e in errs.items():
            assert e <= TOL[prec], (prec, e)
    finally:
        eng.center_to_zero(0)


@pytest.mark.parametrize("bond", [0, 4, 40, 75])
def test_mixed_zero_site_matches_oracle(c1_random, bond):
    p, eng = c1_random
    W = TDVPState.start(p, D=1).W
    mps0 = eng.get_mps(0)                         # centre at 0: sites > bond right-canonical
    R = np.ones((1, 1, 1), complex)
    for j in range(len(mps0) - 1, bond, -1):
        R = env_right(R, mps0[j], W[j])
    eng.move_center(0, bond + 1)
    try:
        mps1 = eng.get_mps(0)                     # sites <= bond left-canonical
        L = np.ones((1, 1, 1), complex)
        for j in range(bond + 1):
            L = env_left(L, mps1[j], W[j])
        Db = mps1[bond].shape[2]
        rng = np.random.default_rng(7 + bond)
        x = rng.normal(size=(Db, Db)) + 1j * rng.normal(size=(Db, Db))
        yo = h0_apply(L, R, x)
        y64 = eng.apply_h0(0, bond, x, precision=pkg.PREC_FP64)
        assert _rel(y64, yo) <= 1e-12
        for prec in (pkg.PREC_TF32, pkg.PREC_TF32X3):
            e = _rel(eng.apply_h0(0, bond, x, precision=prec), yo)
            print(f"bond {bond}: prec {prec} rel err {e:.2e}")
            assert e <= TOL[prec], (prec, e)
    finally:
        eng.center_to_zero(0)


@pytest.mark.parametrize("prec,tol", [(2, 1e-5), (1, 3e-3)])
def test_mixed_steps_track_fp64_oracle(prec, tol):
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
