"""GB300 (sm_103a) spaND + s-step GMRES for the DG Newton-step linear solve.

Public API (all compute in the CUDA library libspand_gb300.so):
    assemble, spmv, Plan, Factor, sstep_gmres, SpandSolve
"""
from .api import BSR, Factor, Plan, assemble, parse_table, spmv, sstep_gmres  # noqa: F401
from ._lib import SpandError  # noqa: F401
