"""FP64 CPU oracle of the F-BMP blind pansharpening method (arXiv 2103.09943).

TEST INFRASTRUCTURE. This package is the plain, slow, obviously-correct
statement of what the CUDA path computes. Only the tests, the smoke check of
``__graft_entry__`` and the benchmark's CPU-baseline / reference arm may import
it; the product path never does, and it shares no code with the CUDA path.

Pins: every function here is checked, in ``tests/test_oracle_*.py``, against
something other than itself (adjoint identities, library routines on special
cases, dense assemblies of the paper's matrices, brute force on tiny inputs,
planted-kernel recovery). Parity is unpinned only for end-to-end quality on
the paper's datasets, which are not available.
"""
from . import fbmp
from ._clib import build
from .fbmp import (PRIORS, apply_z0_prior, apply_zstep_prior, cg_op, filt, filt_adj,
                   guide_stats, prior_filters, prior_stats, solve_band_prior, solve_hrms_prior,
                   HrmsParams, KernelParams, PanStats, admm, apply_z0_system, cg_relchange,
                   apply_zstep_system, bicubic_up, blur_decimate, blur_decimate_adj,
                   box_filter, cg_solve, estimate_kernel, estimate_omega,
                   guided_filter, kernel_error_pct, kernel_normal_eq,
                   jacobi_diag, laplacian, matting_apply, pan_stats, pansharpen,
                   pcg_diag_solve, pcg_solve, precond_apply, psnr, rel_l2, simplex_project, solve_band,
                   solve_hrms, up_solve)

__all__ = [
    "cg_relchange", "PRIORS", "apply_z0_prior", "apply_zstep_prior", "cg_op", "filt",
    "filt_adj", "guide_stats", "prior_filters", "prior_stats", "solve_band_prior",
    "solve_hrms_prior",
    "fbmp", "build", "HrmsParams", "KernelParams", "PanStats", "admm",
    "apply_z0_system", "apply_zstep_system", "bicubic_up", "blur_decimate",
    "blur_decimate_adj", "box_filter", "cg_solve", "estimate_kernel",
    "estimate_omega", "guided_filter", "kernel_error_pct", "kernel_normal_eq",
    "jacobi_diag", "laplacian", "matting_apply", "pan_stats", "pansharpen", "pcg_diag_solve",
    "pcg_solve", "precond_apply", "psnr", "rel_l2",
    "simplex_project", "solve_band", "solve_hrms", "up_solve",
]
