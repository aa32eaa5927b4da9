"""ctypes declarations of the C-ABI in include/ps.h, include/ps_ops.h and
include/ps_cnn.h.

Loading fails loudly when libps.so has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libps.so")


class KernelParams(ctypes.Structure):
    _fields_ = [("lambda_omega", ctypes.c_float), ("l", ctypes.c_int),
                ("alpha1", ctypes.c_float), ("alpha2", ctypes.c_float),
                ("mu1", ctypes.c_float), ("mu2", ctypes.c_float),
                ("mu3", ctypes.c_float), ("rho", ctypes.c_float),
                ("t_max", ctypes.c_int), ("th", ctypes.c_float),
                ("band_mask", ctypes.c_ulonglong)]


class HrmsParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_float), ("r", ctypes.c_int),
                ("eps", ctypes.c_float), ("tol", ctypes.c_float),
                ("max_iter", ctypes.c_int), ("exact_weight", ctypes.c_int),
                ("host_loop", ctypes.c_int), ("precond", ctypes.c_int),
                ("precond_gamma", ctypes.c_float), ("warm", ctypes.c_int),
                ("cnn_params", ctypes.c_void_p), ("stop_rule", ctypes.c_int),
                ("zstep_fp32", ctypes.c_int), ("prior", ctypes.c_int),
                ("precond_diag", ctypes.c_void_p), ("diag_params", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("prec_rows", ctypes.c_int), ("llp_rows", ctypes.c_int),
                ("llp_pf", ctypes.c_int), ("prec_us", ctypes.c_float * 4),
                ("llp_us", ctypes.c_float * 6), ("split", ctypes.c_int),
                ("split_us", ctypes.c_float * 3), ("llp_bands", ctypes.c_int),
                ("llp2_us", ctypes.c_float * 2), ("prec_impl", ctypes.c_int),
                ("prec_impl_us", ctypes.c_float * 2), ("db_impl", ctypes.c_int),
                ("db_impl_us", ctypes.c_float * 2), ("llp_ring_us", ctypes.c_float * 2),
                ("llp_form", ctypes.c_int), ("llp_lean_us", ctypes.c_float * 8)]


class BandInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("ms", ctypes.c_float)]


class KernelInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("last_change", ctypes.c_double)]


class Scene(ctypes.Structure):
    _fields_ = [("lrms", ctypes.c_void_p), ("pan", ctypes.c_void_p),
                ("hrms", ctypes.c_void_p), ("kernel", ctypes.c_void_p),
                ("N", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("ratio", ctypes.c_int), ("R", ctypes.c_int),
                ("band_mask", ctypes.c_ulonglong), ("h_lrms", ctypes.c_void_p),
                ("h_pan", ctypes.c_void_p), ("h_hrms", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_Z = ctypes.c_size_t

# name -> (restype, argtypes); the list is the full exported C-ABI.
SIGNATURES = {
    "ps_default_kernel_params": (None, [ctypes.POINTER(KernelParams)]),
    "ps_default_hrms_params": (None, [ctypes.POINTER(HrmsParams)]),
    "ps_status_string": (ctypes.c_char_p, [_I]),
    "ps_sync_status": (_I, [_P]),
    "ps_workspace_size": (_Z, [_I, _I, _I, _I, _I, _P]),
    "ps_estimate_kernel": (_I, [_P, _P, _I, _I, _I, _I, _I, ctypes.POINTER(KernelParams),
                                _P, _P, _P, ctypes.POINTER(KernelInfo), _P, _Z, _P]),
    "ps_solve_hrms": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, ctypes.POINTER(HrmsParams),
                           _P, _P, _P, _P, _P, _Z, _P]),
    "ps_autotune": (_I, [_I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _Z, _P,
                         ctypes.POINTER(Tuning)]),
    "ps_get_tuning": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(Tuning)]),
    "ps_set_tuning": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(Tuning)]),
    "ps_pansharpen": (_I, [_P, _P, _I, _I, _I, _I, _I, ctypes.POINTER(KernelParams),
                           ctypes.POINTER(HrmsParams), _P, _P, ctypes.POINTER(KernelInfo),
                           _P, _P, _Z, _P]),
    "ps_batch_workspace_size": (_Z, [ctypes.POINTER(Scene), _I, _P]),
    "ps_pansharpen_batched": (_I, [ctypes.POINTER(Scene), _I, _P, ctypes.POINTER(HrmsParams),
                                   _P, _P, _P, _Z, _P]),
    "ps_batch_scene_ms": (_I, [_P, _I, _P, ctypes.POINTER(ctypes.c_double)]),
    "ps_op_blur_decimate": (_I, [_P, _I, _I, _I, _I, _P, _I, _P, _P]),
    "ps_op_blur_decimate_adj": (_I, [_P, _I, _I, _I, _I, _P, _I, _P, _P]),
    "ps_op_pan_stats": (_I, [_P, _I, _I, _I, _F, _P, _P, _P, _P]),
    "ps_op_jacobi_diag": (_I, [_I, _I, _I, _P, _I, _P, _P, _P, _I, _F, _P, _P, _Z, _P]),
    "ps_op_apply_z0": (_I, [_P, _I, _I, _I, _I, _P, _I, _P, _P, _P, _I, _F, _P, _P, _Z, _P]),
    "ps_op_guided_filter": (_I, [_P, _I, _I, _I, _P, _P, _P, _I, _P, _P, _Z, _P]),
    "ps_op_zstep": (_I, [_P, _P, _I, _I, _I, _I, _P, _I, _P, _P, _P, _I, _F, _I, _P, _P, _Z,
                         _P]),
    "ps_op_bicubic_up": (_I, [_P, _I, _I, _I, _I, _P, _P]),
    "ps_cnn_param_count": (_I, []),
    "ps_cnn_workspace_size": (_Z, [_I, _I, _I, _I]),
    "ps_cnn_forward": (_I, [_P, _P, _P, _Z, _I, _I, _I, _P, _P, _Z, _P]),
    "ps_cnn_loss_grad": (_I, [_P, _P, _P, _Z, _P, _I, _I, _I, _P, _P, _P, _Z, _P]),
    "ps_cnn_loss_grad_weighted": (_I, [_P, _P, _P, _Z, _P, _P, _I, _I, _I, _P, _P, _P, _Z, _P]),
    "ps_cnn_adam": (_I, [_P, _P, _P, _P, _I, _F, _F, _F, _F, _P]),
    "ps_cnn_sync_status": (_I, [_P, _I, _I, _I, _I, _P]),
    "ps_op_cnn_conv32": (_I, [_P, _I, _I, _I, _P, _P, _P, _I, _P, _P, _Z, _P]),
    "ps_op_precond": (_I, [_P, _I, _I, _I, _I, _P, _I, _F, _P, _P, _Z, _P]),
    "ps_op_omega": (_I, [_P, _P, _I, _I, _I, _I, _I, _F, _P, _P, _Z, _P]),
    "ps_op_kernel_normal_eq": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P, _P, _P, _Z, _P]),
    "ps_op_admm": (_I, [_P, _P, _I, ctypes.POINTER(KernelParams), _P,
                        ctypes.POINTER(KernelInfo), _P, _Z, _P]),
    "ps_op_workspace_size": (_Z, [_I, _I, _I, _I, _I]),
    "ps_op_kernel_normal_eq_noalloc": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P, _P, _P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libps.so and declare every entry point. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
