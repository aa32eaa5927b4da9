"""Operator-level binding (include/ps_ops.h) on torch CUDA tensors: each step
of the hot path on its own. Marshalling only; the work runs in libps.so."""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from .api import KernelInfo, _check, _f32, _ptr, _stream, default_kernel_params


def _ws(N, H, W, ratio, R, device):
    n = int(_lib.load().ps_op_workspace_size(N, H, W, ratio, R))
    return torch.empty(max(n, 256), dtype=torch.uint8, device=device)


def blur_decimate(z, kernel, ratio):
    """D B(u) z for z of shape (N, H, W)."""
    N, H, W = z.shape
    _f32(z, "z"), _f32(kernel, "kernel")
    out = torch.empty((N, H // ratio, W // ratio), dtype=torch.float32, device=z.device)
    _check(_lib.load().ps_op_blur_decimate(_ptr(z), N, H, W, ratio, _ptr(kernel),
                                           kernel.shape[0] // 2, _ptr(out), _stream()))
    return out


def blur_decimate_adj(v, kernel, ratio):
    """B(u)^T D^T v for v of shape (N, h, w)."""
    N, h, w = v.shape
    _f32(v, "v"), _f32(kernel, "kernel")
    out = torch.empty((N, h * ratio, w * ratio), dtype=torch.float32, device=v.device)
    _check(_lib.load().ps_op_blur_decimate_adj(_ptr(v), N, h * ratio, w * ratio, ratio,
                                               _ptr(kernel), kernel.shape[0] // 2, _ptr(out),
                                               _stream()))
    return out


def pan_stats(pan, r, eps):
    """(I, mu, s) of the PAN (H, W)."""
    H, W = pan.shape
    _f32(pan, "pan")
    I, mu, s = (torch.empty_like(pan) for _ in range(3))
    _check(_lib.load().ps_op_pan_stats(_ptr(pan), H, W, r, ctypes.c_float(eps), _ptr(I),
                                       _ptr(mu), _ptr(s), _stream()))
    return I, mu, s


def apply_z0(z, kernel, ratio, I, mu, s, r, lam):
    """(B^T D^T D B + lam L^T M L) z for z of shape (N, H, W)."""
    N, H, W = z.shape
    for t, nm in ((z, "z"), (kernel, "kernel"), (I, "I"), (mu, "mu"), (s, "s")):
        _f32(t, nm)
    R = kernel.shape[0] // 2
    out = torch.empty_like(z)
    ws = _ws(N, H, W, ratio, R, z.device)
    _check(_lib.load().ps_op_apply_z0(_ptr(z), N, H, W, ratio, _ptr(kernel), R, _ptr(I),
                                      _ptr(mu), _ptr(s), r, ctypes.c_float(lam), _ptr(out),
                                      _ptr(ws), ws.numel(), _stream()))
    return out


def jacobi_diag(kernel, ratio, I, mu, s, r, lam):
    """diag(B^T D^T D B + lam L^T M L) of shape (H, W) (ps_op_jacobi_diag)."""
    H, W = I.shape
    for t, nm in ((kernel, "kernel"), (I, "I"), (mu, "mu"), (s, "s")):
        _f32(t, nm)
    R = kernel.shape[0] // 2
    out = torch.empty((H, W), dtype=torch.float32, device=I.device)
    ws = _ws(1, H, W, ratio, R, I.device)
    _check(_lib.load().ps_op_jacobi_diag(H, W, ratio, _ptr(kernel), R, _ptr(I), _ptr(mu), _ptr(s),
                                         r, ctypes.c_float(lam), _ptr(out), _ptr(ws), ws.numel(),
                                         _stream()))
    return out


def guided_filter(q, I, mu, s, r):
    """Guided filter of q (N, H, W) with guide I."""
    N, H, W = q.shape
    for t, nm in ((q, "q"), (I, "I"), (mu, "mu"), (s, "s")):
        _f32(t, nm)
    out = torch.empty_like(q)
    ws = torch.empty(H * W * 16, dtype=torch.uint8, device=q.device)
    _check(_lib.load().ps_op_guided_filter(_ptr(q), N, H, W, _ptr(I), _ptr(mu), _ptr(s), r,
                                           _ptr(out), _ptr(ws), ws.numel(), _stream()))
    return out


def zstep(lrms, z0, kernel, ratio, I, mu, s, r, lam, exact_weight=False):
    """Z step of Algorithm 2 given Z0 (N, H, W)."""
    N, H, W = z0.shape
    for t, nm in ((lrms, "lrms"), (z0, "z0"), (kernel, "kernel"), (I, "I"), (mu, "mu"),
                  (s, "s")):
        _f32(t, nm)
    R = kernel.shape[0] // 2
    out = torch.empty_like(z0)
    ws = _ws(N, H, W, ratio, R, z0.device)
    _check(_lib.load().ps_op_zstep(_ptr(lrms), _ptr(z0), N, H, W, ratio, _ptr(kernel), R,
                                   _ptr(I), _ptr(mu), _ptr(s), r, ctypes.c_float(lam),
                                   int(exact_weight), _ptr(out), _ptr(ws), ws.numel(),
                                   _stream()))
    return out


def bicubic_up(lrms, ratio):
    """Bicubic x ratio upsampling (Keys, a = -1/2) of (N, h, w) LR bands."""
    N, h, w = lrms.shape
    _f32(lrms, "lrms")
    out = torch.empty((N, h * ratio, w * ratio), dtype=torch.float32, device=lrms.device)
    _check(_lib.load().ps_op_bicubic_up(_ptr(lrms), N, h * ratio, w * ratio, ratio, _ptr(out),
                                        _stream()))
    return out


def cnn_conv32(x, weight, bias=None, mode=0, mask=None):
    """One 32 -> 32 3 x 3 convolution on the tensor cores: x (N, H, W, 32)
    BF16 NHWC, weight (32, 32, 3, 3) FP32. mode 0: ReLU(conv + bias), 1:
    conv + bias, 2: adjoint (backward data), masked by mask > 0 if given."""
    N, H, W, C = x.shape
    if C != 32 or x.dtype != torch.bfloat16 or not x.is_contiguous():
        raise ValueError("x must be contiguous (N, H, W, 32) bfloat16")
    _f32(weight, "weight")
    if bias is not None:
        _f32(bias, "bias")
    out = torch.empty_like(x)
    ws = torch.empty(18688, dtype=torch.uint8, device=x.device)
    _check(_lib.load().ps_op_cnn_conv32(_ptr(x), N, H, W, _ptr(weight),
                                        _ptr(bias) if bias is not None else None,
                                        _ptr(mask) if mask is not None else None, mode,
                                        _ptr(out), _ptr(ws), ws.numel(), _stream()))
    return out


def precond(r, kernel, ratio, lambda_gamma):
    """z = P^{-1} r per band, P = B^T D^T D B + lambda_gamma L^T L (N, H, W)."""
    N, H, W = r.shape
    _f32(r, "r"), _f32(kernel, "kernel")
    R = kernel.shape[0] // 2
    out = torch.empty_like(r)
    ws = _ws(N, H, W, ratio, R, r.device)
    _check(_lib.load().ps_op_precond(_ptr(r), N, H, W, ratio, _ptr(kernel), R,
                                     ctypes.c_float(lambda_gamma), _ptr(out), _ptr(ws),
                                     ws.numel(), _stream()))
    return out


def omega(lrms, pan, ratio, l, lambda_omega):
    N = lrms.shape[0]
    H, W = pan.shape
    _f32(lrms, "lrms"), _f32(pan, "pan")
    out = torch.empty(N, dtype=torch.float32, device=pan.device)
    ws = _ws(N, H, W, ratio, 0, pan.device)
    _check(_lib.load().ps_op_omega(_ptr(lrms), _ptr(pan), N, H, W, ratio, l,
                                   ctypes.c_float(lambda_omega), _ptr(out), _ptr(ws),
                                   ws.numel(), _stream()))
    return out


def kernel_normal_eq(lrms, pan, omega_, ratio, R):
    """(E^T E, E^T f) in float64."""
    N = lrms.shape[0]
    H, W = pan.shape
    _f32(lrms, "lrms"), _f32(pan, "pan"), _f32(omega_, "omega")
    nt = (2 * R + 1) ** 2
    ete = torch.empty((nt, nt), dtype=torch.float64, device=pan.device)
    etf = torch.empty(nt, dtype=torch.float64, device=pan.device)
    ws = _ws(N, H, W, ratio, R, pan.device)
    _check(_lib.load().ps_op_kernel_normal_eq(_ptr(lrms), _ptr(pan), _ptr(omega_), N, H, W,
                                              ratio, R, _ptr(ete), _ptr(etf), _ptr(ws),
                                              ws.numel(), _stream()))
    return ete, etf


def admm(ete, etf, R, params=None):
    """Algorithm 1's loop given E^T E, E^T f (float64). Returns (kernel, info)."""
    if ete.dtype != torch.float64 or etf.dtype != torch.float64:
        raise TypeError("ete and etf must be float64")
    n = 2 * R + 1
    p = params or default_kernel_params()
    kern = torch.empty((n, n), dtype=torch.float32, device=ete.device)
    ws = _ws(1, 4 * n, 4 * n, 2, R, ete.device)
    ki = KernelInfo()
    _check(_lib.load().ps_op_admm(_ptr(ete.contiguous()), _ptr(etf.contiguous()), R,
                                  ctypes.byref(p), _ptr(kern), ctypes.byref(ki), _ptr(ws),
                                  ws.numel(), _stream()))
    return kern, ki


def kernel_normal_eq_noalloc(lrms, pan, omega_, ratio, R):
    """(E^T E, E^T f) like kernel_normal_eq, through the entry point that takes
    no workspace (its scratch is a fixed array owned by the library)."""
    N = lrms.shape[0]
    H, W = pan.shape
    _f32(lrms, "lrms"), _f32(pan, "pan"), _f32(omega_, "omega")
    nt = (2 * R + 1) ** 2
    ete = torch.empty((nt, nt), dtype=torch.float64, device=pan.device)
    etf = torch.empty(nt, dtype=torch.float64, device=pan.device)
    _check(_lib.load().ps_op_kernel_normal_eq_noalloc(_ptr(lrms), _ptr(pan), _ptr(omega_), N, H,
                                                      W, ratio, R, _ptr(ete), _ptr(etf),
                                                      _stream()))
    return ete, etf
