"""GB300-native preconditioned FAS smoothers (AW / ARK with SGS-FVS preconditioning) for
2D finite-volume Euler / thin-layer RANS on structured C-grids.

The compute path is the CUDA library ``libfasw.so`` (C ABI in ``include/fasw.h``);
this package only marshals arguments to it.  There is no CPU fallback.
"""
from .fasw import (FASW_AW3, FASW_AW5J, FASW_AW51, FASW_AW52, FASW_ARK3J, FASW_ARK5J,
                   FASW_ARK51, FASW_ARK52, FASW_FP64, FASW_MIXED, FaswError, Params, Solver,
                   check_math, checkpoint_schedule, default_params, library, library_path, SCHEME_IDS)

__all__ = ["FASW_AW3", "FASW_AW5J", "FASW_AW51", "FASW_AW52", "FASW_ARK3J", "FASW_ARK5J",
           "FASW_ARK51", "FASW_ARK52", "FASW_FP64", "FASW_MIXED", "FaswError", "Params", "Solver",
           "check_math", "checkpoint_schedule", "default_params", "library", "library_path", "SCHEME_IDS"]
