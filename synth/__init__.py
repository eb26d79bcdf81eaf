"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This package only draws inputs: O-grid node coordinates around a NACA-4-digit
shaped curve, modal DG states and solver settings.  It contains none of the
method's arithmetic (no quadrature, no flux, no factorization); both the CPU
oracle and the CUDA library consume what it produces.
"""
from .configs import CONFIGS, Config, get_config  # noqa: F401
from .mesh import naca_ogrid  # noqa: F401
from .state import freestream_conserved, modal_state, uniform_modal_state  # noqa: F401
