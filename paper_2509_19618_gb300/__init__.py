"""GB300-native HPL-MxP solver: low-precision LU without pivoting + fp64
GMRES-based iterative refinement (Dongarra & Luszczek, arXiv 2509.19618).

The compute path is libhpmxp.so (hand-written CUDA for sm_103a, C ABI in
include/hpmxp.h); this package only marshals arguments and uses PyTorch for
device memory and streams.
"""
from . import capi
from .capi import (BF16, FP16, FP8_E4M3, DIAG_DOMINANT, DIAG_SQRTN, DIAG_NONE, HpmxpError, IRInfo, IRParams,
                   hpmxp_factor, hpmxp_factor_workspace, hpmxp_generate, hpmxp_generate_workspace,
                   hpmxp_ir_params_default, hpmxp_residual, hpmxp_residual_workspace, hpmxp_solve_ir,
                   hpmxp_solve_workspace)

__all__ = ["capi", "BF16", "FP16", "FP8_E4M3", "DIAG_DOMINANT", "DIAG_SQRTN", "DIAG_NONE", "HpmxpError",
           "IRInfo", "IRParams", "hpmxp_factor", "hpmxp_factor_workspace", "hpmxp_generate",
           "hpmxp_generate_workspace", "hpmxp_ir_params_default", "hpmxp_residual", "hpmxp_residual_workspace",
           "hpmxp_solve_ir", "hpmxp_solve_workspace"]

