"""Batched ragged realisations (static disorder, ragged bond dims) advanced in the same launches.

Every realisation must follow the trajectory it has when advanced alone: all kernels treat the
realisations independently, only the gauge-shift QR may use a different block count (a different
summation order), so FP64 results agree to rounding and mixed-precision results to the noise of
the tensor-core products.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1907_12044_b300 as pkg  # noqa: E402
from gpu_util import rel_pop_err  # noqa: E402


def _engine(params, Ds, rtol, tune):
    eng = pkg.Engine(n_realisations=len(params))
    eng.set_option(pkg.OPT_RANK_RTOL, rtol)
    for r, (q, D) in enumerate(zip(params, Ds)):
        eng.build_mpo(r, q)
        eng.init_mps(r, D, q.exciton_site)
    if tune:
        eng.autotune()
    return eng


@pytest.mark.parametrize("prec,tol", [(pkg.PREC_FP64, 1e-10), (pkg.PREC_TF32X3, 1e-7)])
def test_batched_fmo_realisations_match_single_runs(prec, tol):
    base = wl.fmo_sized()
    Ds = [32, 64, 48]
    params = [wl.disorder_realisation(base, r) for r in range(3)]
    eng = _engine(params, Ds, 1e-6, tune=True)
    eng.step(10.0, precision=prec)
    for r, (q, D) in enumerate(zip(params, Ds)):
        single = _engine([q], [D], 1e-6, tune=False)
        single.step(10.0, precision=prec)
        Pb = eng.observables(r)[0]
        Ps = single.observables(0)[0]
        assert rel_pop_err(Pb, Ps) <= tol, (r, rel_pop_err(Pb, Ps))
        single.close()



def test_batched_fmo_realisations_match_the_oracle():
    """Two FMO-sized disorder realisations with different bond dimensions in the same launches,
    one FP64 step: each realisation's populations against its own oracle run (<= 1e-10 relative)."""
    from oracle import TDVPState, tdvp_ps_step, populations
    base = wl.fmo_sized()
    Ds = [16, 24]
    params = [wl.disorder_realisation(base, r) for r in (3, 7)]
    eng = _engine(params, Ds, 1e-6, tune=True)
    eng.step(10.0, precision=pkg.PREC_FP64)
    for r, (q, D) in enumerate(zip(params, Ds)):
        st = TDVPState.start(q, D=D)
        tdvp_ps_step(st, 10.0, rank_rtol=1e-6)
        err = rel_pop_err(eng.observables(r)[0], populations(st, q))
        print(f"realisation {r} (D = {D}): relative population error {err:.2e}")
        assert err <= 1e-10
    eng.close()
