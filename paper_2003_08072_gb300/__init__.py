"""GB300 (sm_103a) sketch-preconditioned interior-point LP solver.

Chowdhury, London, Avron & Drineas, "Speeding up Linear Programming using Randomized Linear
Algebra" (arXiv 2003.08072): the infeasible long-step IPM of Algorithm 2 whose normal
equations are solved by the sketch-preconditioned CG of Algorithm 1 with the correction
vector of Eq. compv.  The computation runs in the CUDA library built from ``csrc/`` and is
reached through the C ABI of ``include/lp.h``; this package only marshals arguments.

``LPSolver`` wraps one context for torch tensors (device memory and streams come from
PyTorch); ``LPServer`` drives the library's serving loop (continuous batching of many
instances); the raw entry points are re-exported with their C names.
"""
from __future__ import annotations

from ._binding import (DTYPE_CODES, LP_CSR, LP_DENSE_COLMAJOR, LP_DENSE_ROWMAJOR, LP_BF16,
                       LP_F16, LP_F32, LP_F64, LPError, lp_create, lp_destroy, lp_factor,
                       lp_info, lp_ipm_get_state, lp_ipm_resume, lp_ipm_solve,
                       lp_ipm_state, lp_normal_matvec, lp_normal_solve, lp_params,
                       lp_params_default, lp_profile, lp_profile_enable, lp_profile_read,
                       lp_residuals, lp_set_params, lp_sketch,
                       lp_sketch_indices, lp_step, load, lp_footprint_bytes)
from .server import LPServer
from .solver import LPSolver

__all__ = [
    "LPSolver", "LPError", "load", "lp_params", "lp_info", "lp_params_default", "lp_create",
    "lp_destroy", "lp_set_params", "lp_ipm_solve", "lp_normal_solve", "lp_residuals",
    "lp_sketch_indices", "lp_sketch", "lp_factor", "lp_normal_matvec", "lp_step",
    "LP_DENSE_COLMAJOR", "LP_DENSE_ROWMAJOR", "LP_CSR", "LP_F64", "LP_F32", "LP_BF16", "LP_F16",
    "DTYPE_CODES", "lp_profile", "lp_profile_enable", "lp_profile_read", "LPServer",
    "lp_footprint_bytes", "lp_ipm_state", "lp_ipm_get_state", "lp_ipm_resume",
]
