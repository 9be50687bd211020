"""Seeded synthetic inputs for the Frenkel-Holstein TDVP-PS workloads.

This package is the only code shared by the CPU oracle and the CUDA path.  It
draws model parameters and random start tensors from seeds and holds none of the
time-evolution arithmetic.
"""
from .fh import (FHParams, tiny_chain, fmo_sized, fmo_large, disorder_realisation,
                 ragged_bond_dims, bond_dims, random_mps_tensors, two_level_rabi,
                 single_mode, PHASE_PER_CM_FS)

__all__ = ["FHParams", "tiny_chain", "fmo_sized", "fmo_large", "disorder_realisation",
           "ragged_bond_dims", "bond_dims", "random_mps_tensors", "two_level_rabi",
           "single_mode", "PHASE_PER_CM_FS"]
