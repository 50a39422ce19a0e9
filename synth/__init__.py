"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only draws random numbers and lays them out (integrals, sector
sizes, random isometries for an initial MPS, density-matrix-like test matrices).  It holds none of the DMRG
arithmetic: no Hamiltonian application, no environments, no eigensolvers.
"""
from .integrals import (ab_initio_integrals, hubbard_integrals, config_integrals,
                        batch_problem)
from .mps_gen import (sector_sizes, random_mps, save_mps, load_mps, occupancies)
from .density import TRUNCATION_BATCH_DIMS, graded_density_matrices

__all__ = ["ab_initio_integrals", "hubbard_integrals", "config_integrals", "batch_problem",
           "sector_sizes", "random_mps", "save_mps", "load_mps", "occupancies",
           "TRUNCATION_BATCH_DIMS", "graded_density_matrices"]
