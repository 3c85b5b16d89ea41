"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds geometry and case draws only: C-grid vertex coordinates
around a closed-form NACA 4-digit thickness airfoil, and random case
parameters.  It contains none of the solver's arithmetic (no metrics, fluxes,
boundary conditions or free-stream states); each side computes those itself.
"""
from .cgrid import CGrid, make_cgrid, check_cgrid
from .cases import FlowCase, config_c1, config_c2, config_c3, config_c4_cases, config_c5

__all__ = ["CGrid", "make_cgrid", "check_cgrid", "FlowCase", "config_c1", "config_c2",
           "config_c3", "config_c4_cases", "config_c5"]
