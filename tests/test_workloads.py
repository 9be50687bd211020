"""The synthetic input recipes (seeded stand-ins for the paper's FMO workload, Sec. II.C)."""
import numpy as np

import workloads as wl
from workloads.fh import bond_dims, debye_modes


def test_phase_factor_is_two_pi_c():
    # hbar = 1, energies in cm^-1, times in fs: phase = 2 pi c E t, c = 2.99792458e10 cm/s
    assert abs(wl.PHASE_PER_CM_FS / (2 * np.pi * 2.99792458e10 * 1e-15) - 1.0) < 1e-15


def test_tiny_chain_recipe():
    p = wl.tiny_chain()
    assert p.phys_dims() == [2, 4, 4, 2, 4, 4]
    assert int(np.prod(p.phys_dims())) == 1024
    assert list(p.E) == [12400.0, 12500.0] and p.J[0, 1] == p.J[1, 0] == -80.0
    assert np.allclose(np.concatenate(p.g) ** 2, 0.1) and list(p.omega[0]) == [200.0, 500.0]
    # maximal Schmidt ranks of this chain order (exactness of TDVP at D = 32)
    assert bond_dims(p.phys_dims(), 10 ** 6) == [1, 2, 8, 32, 16, 4, 1]


def test_fmo_sized_and_large_chains():
    p = wl.fmo_sized()
    d = p.phys_dims()
    assert len(d) == 77 and d.count(2) == 7 and d.count(10) == 70
    assert p.el_order == [6, 4, 2, 0, 1, 3, 5]                 # [7,5,3,1,2,4,6], 0-based
    assert [m for kind, m, k in p.chain() if kind == "el"] == p.el_order
    assert np.all((p.E >= 12200) & (p.E <= 12600))
    assert np.allclose(p.J, p.J.T) and np.all(np.diag(p.J) == 0)
    q = wl.fmo_sized()
    assert np.array_equal(p.E, q.E) and np.array_equal(p.J, q.J)
    big = wl.fmo_large()
    d = big.phys_dims()
    assert len(d) == 147 and d.count(16) == 140


def test_debye_discretisation_converges_to_the_cut_continuum():
    """sum_k g_k^2 w_k is a right-endpoint quadrature of (1/pi) int_0^wmax J(w)/w dw, whose closed
    form is (2 lam / pi) atan(wmax / wc); the error is first order in the spacing."""
    lam, wc, wmax = 35.0, 106.0, 500.0
    exact = 2.0 * lam / np.pi * np.arctan(wmax / wc)
    errs = []
    for K in (10, 20, 40):
        w, g = debye_modes(K)
        assert np.allclose(w, wmax / K * np.arange(1, K + 1))
        errs.append(exact - np.sum(g ** 2 * w))
    assert all(e > 0 for e in errs)
    assert abs(errs[0] / errs[1] - 2.0) < 0.05 and abs(errs[1] / errs[2] - 2.0) < 0.05
    w, g = debye_modes(10)
    assert abs(np.sum(g ** 2 * w) - 25.31) < 0.005


def test_disorder_realisations():
    base = wl.fmo_sized()
    reals = [wl.disorder_realisation(base, r) for r in range(256)]
    shifts = np.array([q.E - base.E for q in reals])
    assert abs(shifts.std() / 100.0 - 1.0) < 0.05 and abs(shifts.mean()) < 10.0
    assert all(np.array_equal(q.J, base.J) for q in reals[:5])
    assert not np.array_equal(reals[0].E, reals[1].E)
    assert np.array_equal(wl.disorder_realisation(base, 3).E, reals[3].E)


def test_ragged_draw_is_seeded_and_in_range():
    Ds = wl.ragged_bond_dims(256)
    assert Ds == wl.ragged_bond_dims(256)
    assert set(Ds) <= {32, 48, 64, 96, 128} and len(set(Ds)) == 5
