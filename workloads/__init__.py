"""Seeded synthetic inputs for the Bogacki-Shampine 3(2) coupled-ODE workloads.

This module only draws random numbers with numpy's ``default_rng``.  It holds
none of the solver's arithmetic (no right-hand side, no stage, no error norm),
so both the CPU oracle and the CUDA path may take their inputs from it.
"""

from .generators import (  # noqa: F401
    Workload,
    lco_config,
    lco_paper,
    kuramoto,
    circadian,
    kuramoto_ensemble,
    lco_ragged_batch,
    CIRCADIAN_GLOBALS,
)
