"""Frenkel-Holstein model parameters (Sec. II.C, Eq. holstein) for synthetic workloads.

The paper's FMO parameters come from the literature and an experimental spectral
density (Sec. II.C) that are not available here, so every workload is drawn from a
seed with the sizes of the paper's model: 7 electronic sites, each followed in the
chain by its own vibrational modes, electronic sites ordered [7,5,3,1,2,4,6]
(Sec. II.C), exciton on site 1 at t=0 with all modes in their ground level.

Units: energies and frequencies in cm^-1, times in fs.  With hbar = 1 a phase
E*t picks up the factor 2*pi*c = 1.883651567e-4 rad/(cm^-1 fs).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

# 2*pi*c in rad per (cm^-1 * fs): c = 2.99792458e-5 cm/fs.
PHASE_PER_CM_FS = 2.0 * np.pi * 2.99792458e-5


@dataclass
class FHParams:
    """One Frenkel-Holstein Hamiltonian and its initial product state.

    Electronic sites carry labels 0..n_el-1 (label m is the paper's site m+1).
    ``modes[m]`` lists (omega, g, n_levels) of the modes attached to site m, in the
    order they follow site m along the chain.  ``el_order`` is the chain order of
    the electronic labels.
    """
    E: np.ndarray
    J: np.ndarray
    omega: list
    g: list
    n_levels: list
    el_order: list
    exciton_site: int = 0
    energy_offset: float = 0.0
    include_zpe: bool = False
    name: str = ""

    @property
    def n_el(self) -> int:
        return len(self.E)

    def chain(self):
        """Chain layout: list of (kind, el_label, mode_index), kind in {'el','vib'}."""
        out = []
        for m in self.el_order:
            out.append(("el", m, -1))
            for k in range(len(self.omega[m])):
                out.append(("vib", m, k))
        return out

    def phys_dims(self):
        d = []
        for kind, m, k in self.chain():
            d.append(2 if kind == "el" else int(self.n_levels[m][k]))
        return d

    def occupied(self):
        """Local basis index of the initial product state on every chain site."""
        return [1 if (kind == "el" and m == self.exciton_site) else 0
                for kind, m, k in self.chain()]

    def flat(self):
        """Flattened arrays in the order the C ABI takes them."""
        n_modes = np.array([len(self.omega[m]) for m in range(self.n_el)], dtype=np.int32)
        omega = np.concatenate([np.asarray(self.omega[m], float) for m in range(self.n_el)]) \
            if n_modes.sum() else np.zeros(0)
        g = np.concatenate([np.asarray(self.g[m], float) for m in range(self.n_el)]) \
            if n_modes.sum() else np.zeros(0)
        lev = np.concatenate([np.asarray(self.n_levels[m], np.int32) for m in range(self.n_el)]) \
            if n_modes.sum() else np.zeros(0, np.int32)
        return dict(E=np.asarray(self.E, float), J=np.asarray(self.J, float).reshape(-1),
                    n_modes=n_modes, omega=omega, g=g, n_levels=lev.astype(np.int32),
                    el_order=np.asarray(self.el_order, np.int32))


def bond_dims(d, D):
    """Bond dimensions D_b = min(D, prod of d left of the bond, prod right of it).

    Returns N+1 numbers with 1 at both open ends.
    """
    n = len(d)
    out = [1]
    for b in range(1, n):
        left = 1
        for x in d[:b]:
            left = min(left * x, 1 << 40)
        right = 1
        for x in d[b:]:
            right = min(right * x, 1 << 40)
        out.append(int(min(D, left, right)))
    out.append(1)
    return out


def debye_modes(K, lam=35.0, omega_c=106.0, omega_max=500.0):
    """Equally spaced discretisation of a Debye spectral density (Sec. II.C).

    J(w) = 2 lam w w_c / (w^2 + w_c^2); w_k = k dw, dw = omega_max / K;
    g_k^2 = J(w_k) dw / (pi w_k^2), so that sum_k g_k^2 w_k approximates lam.
    """
    if K == 0:
        return np.zeros(0), np.zeros(0)
    dw = omega_max / K
    w = dw * np.arange(1, K + 1)
    Jw = 2.0 * lam * w * omega_c / (w * w + omega_c * omega_c)
    g = np.sqrt(Jw * dw / (np.pi * w * w))
    return w, g


def tiny_chain():
    """Two electronic sites, two modes each, 4 phonon levels: 6 chain sites, dim 1024."""
    E = np.array([12400.0, 12500.0])
    J = np.array([[0.0, -80.0], [-80.0, 0.0]])
    w = np.array([200.0, 500.0])
    g = np.full(2, np.sqrt(0.1))
    return FHParams(E=E, J=J, omega=[w, w.copy()], g=[g, g.copy()],
                    n_levels=[np.array([4, 4]), np.array([4, 4])], el_order=[0, 1],
                    exciton_site=0, energy_offset=float(E.mean()), name="tiny-2site")


def _fmo_energies(seed):
    rng = np.random.default_rng(seed)
    E = rng.uniform(12200.0, 12600.0, size=7)
    J = np.zeros((7, 7))
    for m in range(7):
        for n in range(m + 1, 7):
            J[m, n] = J[n, m] = rng.normal(0.0, 40.0)
    return E, J


FMO_ORDER = [6, 4, 2, 0, 1, 3, 5]


def fmo_sized(n_modes=10, n_levels=10, seed=1907):
    """FMO-sized chain: 7 sites, ``n_modes`` Debye modes each (77 sites for 10)."""
    E, J = _fmo_energies(seed)
    w, g = debye_modes(n_modes)
    return FHParams(E=E, J=J, omega=[w.copy() for _ in range(7)], g=[g.copy() for _ in range(7)],
                    n_levels=[np.full(n_modes, n_levels) for _ in range(7)], el_order=list(FMO_ORDER),
                    exciton_site=0, energy_offset=float(E.mean()),
                    name=f"fmo-7x{n_modes}-L{n_levels}")


def fmo_large():
    """The 147-site chain: 20 modes per electronic site, 16 levels."""
    return fmo_sized(n_modes=20, n_levels=16)


def disorder_realisation(base: FHParams, r: int, sigma=100.0, seed=1907):
    """Static disorder: site energies of ``base`` plus N(0, sigma^2), seed seed+1+r."""
    rng = np.random.default_rng(seed + 1 + r)
    E = base.E + rng.normal(0.0, sigma, size=base.n_el)
    return FHParams(E=E, J=base.J.copy(), omega=[x.copy() for x in base.omega],
                    g=[x.copy() for x in base.g], n_levels=[x.copy() for x in base.n_levels],
                    el_order=list(base.el_order), exciton_site=base.exciton_site,
                    energy_offset=float(base.energy_offset), name=f"{base.name}-dis{r}")


def ragged_bond_dims(n, choices=(32, 48, 64, 96, 128), seed=12044):
    """Per-realisation bond dimension drawn uniformly from ``choices``."""
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.choice(np.asarray(choices), size=n)]


def two_level_rabi(E1=12400.0, E2=12500.0, J=-80.0):
    """Two electronic sites and no modes (closed-form Rabi oscillation)."""
    E = np.array([E1, E2])
    Jm = np.array([[0.0, J], [J, 0.0]])
    return FHParams(E=E, J=Jm, omega=[np.zeros(0), np.zeros(0)], g=[np.zeros(0), np.zeros(0)],
                    n_levels=[np.zeros(0, int), np.zeros(0, int)], el_order=[0, 1],
                    exciton_site=0, energy_offset=float(E.mean()), name="rabi")


def single_mode(omega=200.0, S=0.1, levels=12):
    """One electronic site with one mode, exciton present (displaced oscillator)."""
    E = np.array([12400.0])
    return FHParams(E=E, J=np.zeros((1, 1)), omega=[np.array([omega])], g=[np.array([np.sqrt(S)])],
                    n_levels=[np.array([levels])], el_order=[0], exciton_site=0,
                    energy_offset=12400.0, name="single-mode")


def random_mps_tensors(d, D, seed=7):
    """Seeded complex Gaussian site tensors [Dl, d, Dr] at the bond dims of ``bond_dims``.

    Generic (full-rank with probability one), not canonical and not normalised.
    """
    rng = np.random.default_rng(seed)
    bd = bond_dims(d, D)
    out = []
    for i, di in enumerate(d):
        shape = (bd[i], di, bd[i + 1])
        out.append(rng.normal(size=shape) + 1j * rng.normal(size=shape))
    return out
