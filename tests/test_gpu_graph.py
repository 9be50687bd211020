"""Whole steps replayed as a CUDA graph (one conditional while node per Lanczos exponential)
against the launch-by-launch path and the oracle.

With the convergence test at every k both paths run the same kernels on the same data in the same
order, so their results must be identical bit for bit; the graph path also matches the CPU oracle
like the launch-by-launch path does.
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
from gpu_util import rel_pop_err  # noqa: E402

POP_TOL = 1e-10


def make(p, D, graph, R=1, dims=None, params=None):
    eng = pkg.Engine(n_realisations=R)
    eng.set_option(pkg.OPT_KRYLOV_CHECK_ALL, 1)
    eng.set_option(pkg.OPT_GRAPH, 1 if graph else 0)
    for r in range(R):
        q = params[r] if params else p
        eng.build_mpo(r, q)
        eng.init_mps(r, dims[r] if dims else D, q.exciton_site)
    return eng


@pytest.mark.parametrize("prec", [pkg.PREC_FP64, pkg.PREC_TF32X3])
def test_graph_steps_equal_launch_by_launch_tiny(prec):
    p = wl.tiny_chain()
    a, b = make(p, 16, False), make(p, 16, True)
    st = TDVPState.start(p, D=16)
    for _ in range(6):
        a.step(10.0, precision=prec)
        b.step(10.0, precision=prec)
        Pa, Ea, na = a.observables(0)
        Pb, Eb, nb = b.observables(0)
        assert np.array_equal(Pa, Pb) and Ea == Eb and na == nb
        if prec == pkg.PREC_FP64:
            tdvp_ps_step(st, 10.0)
            assert rel_pop_err(Pb, populations(st, p)) <= POP_TOL
    sa, sb = a.stats(), b.stats()
    assert sa["krylov_solves"] == sb["krylov_solves"]
    assert sa["krylov_dim_sum"] == sb["krylov_dim_sum"]
    assert sb["host_syncs"] < sa["host_syncs"]


def test_graph_multi_step_call_and_recapture_on_new_dt():
    p = wl.tiny_chain()
    a, b = make(p, 8, False), make(p, 8, True)
    a.step(10.0, n_steps=4)
    b.step(10.0, n_steps=4)          # one capture, four replays
    assert np.array_equal(a.observables(0)[0], b.observables(0)[0])
    a.step(5.0, n_steps=2)
    b.step(5.0, n_steps=2)           # new dt: captured again
    assert np.array_equal(a.observables(0)[0], b.observables(0)[0])
    b.set_option(pkg.OPT_GRAPH, 0)   # back to launch by launch on the same state
    a.step(10.0)
    b.step(10.0)
    assert np.array_equal(a.observables(0)[0], b.observables(0)[0])


def test_graph_fmo_sized_mixed_precision_equals_launch_by_launch():
    p = wl.fmo_sized()
    a, b = make(p, 32, False), make(p, 32, True)
    for _ in range(2):
        a.step(10.0, precision=pkg.PREC_TF32X3)
        b.step(10.0, precision=pkg.PREC_TF32X3)
    assert np.array_equal(a.observables(0)[0], b.observables(0)[0])


def test_graph_batched_ragged_realisations_equal_launch_by_launch():
    base = wl.fmo_sized()
    R = 3
    params = [wl.disorder_realisation(base, r) for r in range(R)]
    dims = [16, 32, 24]
    a = make(base, None, False, R=R, dims=dims, params=params)
    b = make(base, None, True, R=R, dims=dims, params=params)
    for _ in range(2):
        a.step(10.0)
        b.step(10.0)
    for r in range(R):
        assert np.array_equal(a.observables(r)[0], b.observables(r)[0])


def test_graph_with_device_side_convergence_start_matches_oracle():
    """Default policy: tests start at the previous Krylov dimension minus 2, kept on the device."""
    p = wl.tiny_chain()
    eng = pkg.Engine()
    eng.set_option(pkg.OPT_GRAPH, 1)
    eng.build_mpo(0, p)
    eng.init_mps(0, 16, p.exciton_site)
    st = TDVPState.start(p, D=16)
    for _ in range(5):
        eng.step(10.0)
        tdvp_ps_step(st, 10.0)
        assert rel_pop_err(eng.observables(0)[0], populations(st, p)) <= POP_TOL
