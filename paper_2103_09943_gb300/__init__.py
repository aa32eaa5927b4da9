"""GB300 (sm_103a) implementation of the hot path of F-BMP blind
multi-spectral pansharpening (arXiv 2103.09943): the TGV^2 blur-kernel
estimate (Algorithm 1) and the per-band HRMS solve under the local
Laplacian prior (Algorithm 2), as hand-written CUDA behind the C-ABI of
include/ps.h and include/ps_ops.h.

The compute runs only in libps.so; importing a function that needs it raises
if the library has not been built.
"""
from .api import (HostPipeline, PsError, default_hrms_params, default_kernel_params,
                  estimate_kernel, pansharpen, solve_hrms, workspace, workspace_size)

__all__ = ["HostPipeline", "PsError", "default_hrms_params", "default_kernel_params",
           "estimate_kernel", "pansharpen", "solve_hrms", "workspace", "workspace_size"]
