"""TDVP-PS on the device from the paper's own kind of initial state.

The paper starts its TDVP runs from a P&C-RK4 warm-up (Sec. II.C; Sec. II.A.1, Eq. RK4): the
Hartree product state propagated for ten 80 a.u. steps by global RK4 with SVD compression, then
compressed to the run's bond dimension.  The oracle computes that state from the product start
(`oracle.pc_rk4`, pinned in `tests/test_oracle_pc_rk4.py`); the final compression also drops
singular values below 1e-8 of the norm (criterion ii of Eq. SVD), so that no bond carries
directions at the level of the gauge shift's rank threshold.  Both sides then run TDVP-PS from
these tensors: no completion of an empty basis is involved anywhere on this path.

Bounds: the FP64 path as in the other whole-step parity tests (relative populations 1e-10,
energy 1e-9); TF32x3 at the mixed-step bound of 1e-5.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import TDVPState, tdvp_ps_step, populations, energy
from oracle.pc_rk4 import warmup, compress

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1907_12044_b300 as pkg  # noqa: E402
from gpu_util import engine_for, rel_pop_err  # noqa: E402

CASES = {
    # chain, M_S, M_max of the warm-up, TDVP steps
    "tiny": (wl.tiny_chain, 8, 64, 20),
    "fmo77": (wl.fmo_sized, 8, 8, 3),
}


@pytest.fixture(scope="module", params=list(CASES))
def warm_start(request):
    maker, M_S, M_max, steps = CASES[request.param]
    p = maker()
    tens = compress(warmup(p, M_S=M_S, M_max=M_max), M_S, zeta=1e-8)
    assert max(A.shape[2] for A in tens) == M_S and min(A.shape[2] for A in tens[:-1]) >= 2
    # the device's shape rules for explicit tensors: Dl <= d Dr and Dr <= Dl d at every site
    assert all(A.shape[0] <= A.shape[1] * A.shape[2] and A.shape[2] <= A.shape[0] * A.shape[1]
               for A in tens)
    return request.param, p, tens, steps


def test_fp64_steps_from_the_warmup_state_match_the_oracle(warm_start):
    name, p, tens, steps = warm_start
    eng = engine_for(p, tensors=tens)
    st = TDVPState.start(p, tensors=tens)
    P, E, nrm = eng.observables(0)
    assert rel_pop_err(P, populations(st, p)) <= 1e-12 and abs(nrm - 1.0) <= 1e-12
    worst = 0.0
    for _ in range(steps):
        eng.step(10.0)
        tdvp_ps_step(st, 10.0)
        P, E, nrm = eng.observables(0)
        worst = max(worst, rel_pop_err(P, populations(st, p)))
        assert abs(E - energy(st)) <= 1e-9 * max(1.0, abs(energy(st)))
    print(f"{name}: warm-up start, {steps} FP64 steps, worst relative population error {worst:.1e}")
    assert worst <= 1e-10
    eng.close()


def test_tf32x3_step_from_the_warmup_state_tracks_the_oracle(warm_start):
    name, p, tens, _ = warm_start
    eng = engine_for(p, tensors=tens)
    st = TDVPState.start(p, tensors=tens)
    eng.step(10.0, precision=pkg.PREC_TF32X3, tol=1e-10)
    tdvp_ps_step(st, 10.0)
    err = rel_pop_err(eng.observables(0)[0], populations(st, p))
    print(f"{name}: warm-up start, one TF32x3 step, relative population error {err:.1e}")
    assert err <= 1e-5
    eng.close()
