"""The fused Lanczos iteration (one cooperative launch per iteration after the matvec) against the
four-launch form, and the bounded waits of its group barriers.

The fused kernel performs the arithmetic of the four kernels in the same order on the same
chunks, so whole steps agree bit for bit.  Its phases are separated by group barriers whose waits
are bounded by wall-clock time; the stall test makes one barrier wait for a block that does not
exist, so the waits run out, the step reports TDVP_ERR_DEVICE_TIMEOUT and the context remains
usable.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import TDVPState, tdvp_ps_step, populations

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1907_12044_b300 as pkg  # noqa: E402
from gpu_util import engine_for, rel_pop_err  # noqa: E402


def _run(p, prec, fused, graph, steps=2, D=64):
    eng = pkg.Engine()
    eng.set_option(pkg.OPT_FUSED_LANCZOS, 1 if fused else 0)
    eng.set_option(pkg.OPT_RANK_RTOL, 1e-6)
    eng.set_option(pkg.OPT_GRAPH, 1 if graph else 0)
    eng.build_mpo(0, p)
    eng.init_mps(0, D, p.exciton_site)
    for _ in range(steps):
        eng.step(10.0, precision=prec, tol=1e-10)
    out = (eng.observables(0)[0], [eng.get_site(0, i) for i in (0, 5, 40)], eng.stats())
    eng.close()
    return out


@pytest.mark.parametrize("prec,graph", [(pkg.PREC_FP64, False), (pkg.PREC_TF32X3, True),
                                        (pkg.PREC_BF16X3, False)])
def test_fused_iteration_is_bit_identical_to_four_launches(prec, graph):
    p = wl.fmo_sized()
    Pa, Sa, sta = _run(p, prec, True, graph)
    Pb, Sb, stb = _run(p, prec, False, graph)
    assert np.array_equal(Pa, Pb)
    for a, b in zip(Sa, Sb):
        assert np.array_equal(a, b)
    # fewer launches per site update with the fused iteration
    assert sta["kernel_launches"] < stb["kernel_launches"]
    print(f"prec {prec} graph {graph}: launches per site update fused "
          f"{sta['kernel_launches'] / sta['site_updates']:.1f}, four-launch "
          f"{stb['kernel_launches'] / stb['site_updates']:.1f}")


def test_stall_test_reports_device_timeout_and_the_context_stays_usable():
    p = wl.tiny_chain()
    eng = engine_for(p, D=8)
    eng.set_option(pkg.OPT_STALL_TEST, 0.01)
    with pytest.raises(pkg.TDVPError) as e:
        eng.step(10.0)
    assert e.value.code == -5
    # the failure is reported once; the same context then runs a normal step from a new start
    eng.set_option(pkg.OPT_STALL_TEST, 0.0)
    eng.init_mps(0, 8, p.exciton_site)
    eng.step(10.0)
    st = TDVPState.start(p, D=8)
    tdvp_ps_step(st, 10.0)
    assert rel_pop_err(eng.observables(0)[0], populations(st, p)) <= 1e-10
    eng.close()


def test_autotuned_tensor_core_splits_keep_mixed_steps_on_the_oracle():
    """The autotuner's split-K choice for every Lanczos-matvec GEMM shape changes only the FP32
    summation order: two TF32x3 steps stay on the FP64 oracle within the mixed-precision bound."""
    p = wl.fmo_sized()
    eng = engine_for(p, D=64)
    eng.set_option(pkg.OPT_RANK_RTOL, 1e-6)
    eng.autotune()
    st = TDVPState.start(p, D=64)
    for _ in range(2):
        eng.step(10.0, precision=pkg.PREC_TF32X3, tol=1e-10)
        tdvp_ps_step(st, 10.0, rank_rtol=1e-6)
    assert rel_pop_err(eng.observables(0)[0], populations(st, p)) <= 1e-5
    eng.close()
