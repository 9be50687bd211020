"""CPU oracle for one-site TDVP projector-splitting (TDVP-PS), complex128.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package: only
the tests, the smoke check in ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` call it.  It shares no code with the CUDA path; the one common input
is the seeded parameter generator in ``workloads``.

Every function is plain numpy/scipy written from the paper's definitions
(Li, Ren, Shuai, arXiv:1907.12044): the MPS gauge and QR (Eq. mix-canon, Eq. QR),
the P&C-RK4 warm-up (Eq. mpo-apply, Eq. mps+mps, Eq. SVD, Eq. RK4; ``pc_rk4``),
the two-site TDVP-PS with SVD truncation (end of Sec. II.A.2; ``tdvp2``), TDVP-MU with the
matrix-unfolding regularisation and CMF (Eq. tdvp1_C, tdvp1_L, tdvp1_mu_L, reg2; ``tdvp_mu``),
the MPO (Eq. mpo), the environments and effective Hamiltonian (Eq. tdvp1_H,
tdvp1_h1i, tdvp1_hiN, tdvp1_h), the TDVP-PS split (Eq. ps_trotter, Eq. tdvp2_C,
Eq. tdvp2_D), the Lanczos exponential (Sec. II.A.2, TDVP-PS paragraph) and the
population error (Eq. error).  Where the paper is silent the reading taken is
stated in the docstring of the function that takes it.

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
against closed forms, dense linear algebra, invariants or brute force.
"""
from .mpo import build_mpo, mpo_to_dense, local_operators
from .linalg import qr_rr, lq_rr, expm_tridiag_e1, lanczos_expm
from .mps import (product_mps, canonicalize_right, heff_apply, h0_apply, env_left, env_right,
                  mps_to_dense)
from .tdvp import TDVPState, tdvp_ps_step, populations, energy, norm, mean_cumulative_deviation
from .pc_rk4 import mpo_apply, mps_add, canonicalise_left, svd_compress, compress, rk4_step, warmup
from .tdvp2 import heff2_apply, truncated_svd, tdvp2_step
from .tdvp_mu import left_canonicalise, regularise, mean_fields, derivative, tdvp_mu_step

__all__ = ["build_mpo", "mpo_to_dense", "local_operators", "qr_rr", "lq_rr", "expm_tridiag_e1",
           "lanczos_expm", "product_mps", "canonicalize_right", "heff_apply", "h0_apply",
           "env_left", "env_right", "mps_to_dense", "TDVPState", "tdvp_ps_step", "populations",
           "energy", "norm", "mean_cumulative_deviation", "mpo_apply", "mps_add", "canonicalise_left",
           "svd_compress", "compress", "rk4_step", "warmup", "heff2_apply", "truncated_svd", "tdvp2_step",
           "left_canonicalise", "regularise", "mean_fields", "derivative", "tdvp_mu_step"]
