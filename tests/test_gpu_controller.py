"""Learned Krylov controller: GPU training kernels against the reference MLP, and its gain.

The controller decides where the convergence tests of a Lanczos exponential start (its predicted
dimension, one later when its acceptance head predicts a failed test there); the a-posteriori
estimate and tolerance still decide where it stops.  Its gain is counted in tridiagonal
exponentials (convergence tests) against the library's default rule (tests from the previous
Krylov dimension of the same site minus 2) and against testing at every k, with the populations
unchanged.  The bench measures the same comparison in wall time.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import mlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1907_12044_b300 as pkg  # noqa: E402
from gpu_util import engine_for, rel_pop_err  # noqa: E402


@pytest.mark.parametrize("head", [0, 1])
def test_gpu_gradients_match_reference_mlp(head):
    eng = pkg.Engine()
    w = mlp.init(5)
    eng.controller_set_weights(w)
    rng = np.random.default_rng(6 + head)
    X = rng.normal(size=(333, mlp.NIN))
    t = rng.uniform(2, 20, size=333) if head == 0 else rng.integers(1, 9, size=333).astype(float)
    loss, g = eng.controller_loss_grad(X, t, head=head)
    f32 = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)
    L_ref, g_ref = mlp.loss_and_grad(f32(w), f32(X), f32(t), head=head)
    assert abs(loss - L_ref) <= 1e-5 * L_ref
    assert np.linalg.norm(g - g_ref) <= 1e-5 * np.linalg.norm(g_ref)
    if head == 1:
        assert np.all(g[:mlp.NPARAM - 65] == 0)
    assert np.allclose(eng.controller_get_weights(), w.astype(np.float32))


def _run(eng, steps, mode):
    pops = []
    for _ in range(steps):
        eng.step(10.0, krylov_mode=mode)
        pops.append(eng.observables(0)[0])
    return np.array(pops)


def test_trained_controller_reduces_convergence_tests_without_changing_results():
    p = wl.fmo_sized()
    # the plain method: convergence tested at every k; its own solves are the training data
    plain = engine_for(p, D=64)
    plain.set_option(pkg.OPT_KRYLOV_CHECK_ALL, 1)
    plain.controller_logging(200000)
    plain.reset_stats()
    P_plain = _run(plain, 3, pkg.KRYLOV_ADAPTIVE)
    tests_plain = plain.stats()["tri_evals"]
    log = plain.controller_log()
    assert log.shape[0] == plain.stats()["krylov_solves"]
    # train on the GPU (Adam): the dimension head, then the acceptance head
    plain.controller_set_weights(mlp.init(0))
    l0 = plain.controller_train(epochs=1, batch=256, lr=1e-3)
    l1 = plain.controller_train(epochs=150, batch=256, lr=3e-3)
    print(f"controller loss (k MSE, acceptance): first epoch {l0}, after training {l1}, samples {log.shape[0]}")
    assert l1[0] < 0.3 * l0[0]
    assert l1[1] < 0.6931                     # better than chance (log 2) on the acceptance labels
    w = plain.controller_get_weights()
    # the library's default rule (tests from the previous dimension minus 2), same start
    default = engine_for(p, D=64)
    default.reset_stats()
    P_default = _run(default, 3, pkg.KRYLOV_ADAPTIVE)
    tests_default = default.stats()["tri_evals"]
    # the same steps with the trained controller
    learned = engine_for(p, D=64)
    learned.controller_set_weights(w)
    learned.reset_stats()
    P_learned = _run(learned, 3, pkg.KRYLOV_LEARNED)
    tests_learned = learned.stats()["tri_evals"]
    print(f"convergence tests: every k {tests_plain}, default rule {tests_default}, learned {tests_learned}")
    assert tests_learned < 0.6 * tests_plain
    assert tests_learned < tests_default
    for a, b, c in zip(P_learned, P_plain, P_default):
        assert rel_pop_err(a, b) <= 1e-9
        assert rel_pop_err(c, b) <= 1e-9
