"""GB300 (sm_103a) spaND + s-step GMRES for the DG Newton-step linear solve.

Public API (all compute in the CUDA library libspand_gb300.so):
    assemble, spmv, Plan, Factor, sstep_gmres, gmres (Algorithm 1 baseline), SpandSolve,
    matrix_powers (the s-step basis with the preconditioner fused into the SpMV chain),
    factor_batched, sstep_gmres_batched (many independent systems),
    march, cfl_ramp (pseudo-time continuation around the solve)
"""
from .api import (BSR, Factor, Plan, SpandSolve, assemble, cfl_ramp, factor_batched, gmres,  # noqa: F401
                  kernel_launches, march, matrix_powers, parse_table, pattern_outer, spmv, sstep_gmres,
                  sstep_gmres_batched)
from ._lib import SpandError  # noqa: F401
