"""Binding of the learned warm start (include/ps_cnn.h) on torch CUDA tensors:
argument marshalling, parameter initialisation and checkpoints. Every
forward, backward and optimizer step runs in libps.so."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .api import _check, _f32, _ptr, _stream

WIDTHS = (2, 32, 32, 32, 32, 32, 1)


def param_count() -> int:
    return int(_lib.load().ps_cnn_param_count())


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (9 in))), zero biases; the last layer
    scaled by 0.1 so that the untrained network returns about its bicubic
    input. Layout: per layer, weights (out, in, 3, 3) then biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(WIDTHS) - 1):
        ci, co = WIDTHS[l], WIDTHS[l + 1]
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if l == len(WIDTHS) - 2 else 1.0)
        parts.append((rng.standard_normal((co, ci, 3, 3)) * std).ravel())
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def split_params(p: np.ndarray):
    """The flat vector as [(w, b), ...] per layer."""
    out, o = [], 0
    for l in range(len(WIDTHS) - 1):
        ci, co = WIDTHS[l], WIDTHS[l + 1]
        w = p[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = p[o:o + co]
        o += co
        out.append((w, b))
    return out


class WarmStartNet:
    """Parameters, Adam moments and workspaces of the warm-start network."""

    def __init__(self, params=None, seed: int = 0, device=None):
        self.device = torch.device(device or "cuda")
        p = init_params(seed) if params is None else np.asarray(params, dtype=np.float32)
        if p.size != param_count():
            raise ValueError(f"expected {param_count()} parameters, got {p.size}")
        self.params = torch.from_numpy(p.copy()).to(self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.step = 0
        self._ws = {}

    def _workspace(self, B, H, W, training):
        key = (B, H, W, training)
        if key not in self._ws:
            n = int(_lib.load().ps_cnn_workspace_size(B, H, W, training))
            if n == 0:
                raise ValueError("invalid sizes")
            self._ws = {key: torch.empty(n, dtype=torch.uint8, device=self.device)}
        return self._ws[key]

    @staticmethod
    def _pan_stride(pan, B, H, W):
        if pan.dim() == 2:
            return 0
        if pan.shape[0] != B:
            raise ValueError("pan must be (H, W) or (B, H, W)")
        return H * W

    def forward(self, up, pan, out=None, check=False):
        """z (B, H, W) from the bicubic upsampling `up` (B, H, W) and the PAN
        ((H, W) shared, or (B, H, W))."""
        B, H, W = up.shape
        _f32(up, "up"), _f32(pan, "pan")
        z = out if out is not None else torch.empty_like(up)
        ws = self._workspace(B, H, W, 0)
        lib = _lib.load()
        _check(lib.ps_cnn_forward(_ptr(self.params), _ptr(up), _ptr(pan),
                                  self._pan_stride(pan, B, H, W), B, H, W, _ptr(z), _ptr(ws),
                                  ws.numel(), _stream()))
        if check:
            _check(lib.ps_cnn_sync_status(_ptr(ws), B, H, W, 0, _stream()))
        return z

    def loss_grad(self, up, pan, target, weight=None):
        """Mean squared error of z / 255 against target / 255 (per-pixel
        weighted when `weight` (B, H, W) is given) and its gradient (into
        self.grad). Returns the loss as a float (synchronises)."""
        B, H, W = up.shape
        _f32(up, "up"), _f32(pan, "pan"), _f32(target, "target")
        ws = self._workspace(B, H, W, 1)
        lib = _lib.load()
        if weight is None:
            _check(lib.ps_cnn_loss_grad(_ptr(self.params), _ptr(up), _ptr(pan),
                                        self._pan_stride(pan, B, H, W), _ptr(target), B, H, W,
                                        _ptr(self.grad), _ptr(self.loss), _ptr(ws), ws.numel(),
                                        _stream()))
        else:
            _f32(weight, "weight")
            if tuple(weight.shape) != (B, H, W):
                raise ValueError("weight must be shaped like up")
            _check(lib.ps_cnn_loss_grad_weighted(_ptr(self.params), _ptr(up), _ptr(pan),
                                                 self._pan_stride(pan, B, H, W), _ptr(target),
                                                 _ptr(weight), B, H, W, _ptr(self.grad),
                                                 _ptr(self.loss), _ptr(ws), ws.numel(),
                                                 _stream()))
        _check(lib.ps_cnn_sync_status(_ptr(ws), B, H, W, 1, _stream()))
        return float(self.loss.item()) / (B * H * W)

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        _check(_lib.load().ps_cnn_adam(_ptr(self.params), _ptr(self.grad), _ptr(self.m),
                                       _ptr(self.v), self.step, ctypes.c_float(lr),
                                       ctypes.c_float(beta1), ctypes.c_float(beta2),
                                       ctypes.c_float(eps), _stream()))

    # checkpoints: weights, Adam moments and the step count
    def save(self, path):
        np.savez(path, params=self.params.cpu().numpy(), m=self.m.cpu().numpy(),
                 v=self.v.cpu().numpy(), step=np.array(self.step))

    @classmethod
    def load(cls, path, device=None):
        d = np.load(path)
        net = cls(params=d["params"], device=device)
        if "m" in d:
            net.m.copy_(torch.from_numpy(d["m"]))
            net.v.copy_(torch.from_numpy(d["v"]))
            net.step = int(d["step"])
        return net
