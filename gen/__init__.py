"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package only *produces inputs*: the shell-model problem of Eq. (1) (single-particle
energies and antisymmetrised m-scheme two-body matrix elements drawn from a J-coupled
random ensemble), the frozen orbital ordering, and the random right-canonical starting
MPS.  It holds none of the DMRG method's arithmetic (no operator algebra, no
eigensolver, no truncation); both the oracle and the CUDA library consume what it
produces as plain arrays.
"""
from .prng import SplitMix64
from .shell import (SPACES, Orbital, Space, Problem, make_problem, cg, site_table,
                    count_sector_dims, mscheme_dimension, pairing_problem)
from .mps import initial_mps, InitialMPS

__all__ = ["SplitMix64", "SPACES", "Orbital", "Space", "Problem", "make_problem", "cg",
           "site_table", "count_sector_dims", "mscheme_dimension", "pairing_problem",
           "initial_mps", "InitialMPS"]
