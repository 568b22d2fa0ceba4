"""Test infrastructure: the CPU oracle of the ISM pressure solve.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It shares no code with the CUDA library.
"""
from .ism_oracle import (OracleISM, OracleACMV, OracleAccommodative, build, lib, apply_af, residual, rbgs_sweep,
                         restrict, prolong_add, prolong_const_add,
                         coarse_operator, coarse_operator_sparse, predictor, divergence, correct,
                         proj_step, VEL_NOSLIP, VEL_FREESLIP, VEL_INFLOW,
                         VEL_OUTFLOW, VEL_PERIODIC, pressure_bc, BC_NEUMANN, BC_DIRICHLET0,
                         BC_PERIODIC, is_singular, periodic_axes, ncoarse, set_threads, get_threads)

__all__ = ["OracleISM", "OracleACMV", "OracleAccommodative", "build", "lib", "apply_af", "residual", "rbgs_sweep",
           "restrict", "prolong_add", "prolong_const_add", "coarse_operator", "coarse_operator_sparse",
           "predictor", "divergence", "correct", "proj_step", "VEL_NOSLIP",
           "VEL_FREESLIP", "VEL_INFLOW", "VEL_OUTFLOW", "VEL_PERIODIC", "pressure_bc",
           "BC_NEUMANN", "BC_DIRICHLET0", "BC_PERIODIC", "is_singular", "periodic_axes", "ncoarse",
           "set_threads", "get_threads"]
