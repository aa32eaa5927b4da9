"""A synthetic analogue of the paper's kernel-prior experiment (Sec. IV-B,
Table II): the kernel of Appendix B with the paper's parameters (R = 9,
centre (1.392, 0.093), sigma = 2, motion d = 3 at -13.7 degrees) blurs a PAN
image, which is decimated by 4 and given white noise at 10..50 dB PSNR (Eq.
psnr_def against the blurred image); Algorithm 1 estimates the kernel from
the noisy measurement and the PAN. The GPU must give the oracle's kernel at
every noise level, and the relative error of Eq. relative_error_kernel must
fall as the PSNR rises. (The paper's own numbers come from a satellite image
that is not available here; they are not the bar.)"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
import synth
from synth.scenes import _motion_kernel
from paper_2103_09943_gb300 import api
from tests.gpu_util import rel, to_np

pytestmark = pytest.mark.gpu


def planted(psnrs, seed=5):
    sc = synth.make_scene(replace(synth.CONFIGS["c1"], H=512, W=512, shapes=60, seed=77))
    Y = sc["pan"].astype(np.float64)
    u = _motion_kernel(9, 1.392, 0.093, 2.0, 3.0, np.deg2rad(-13.7))
    H, W = Y.shape
    k = np.zeros((H, W))
    for i in range(-9, 10):
        for j in range(-9, 10):
            k[i % H, j % W] += u[i + 9, j + 9]
    blur = np.real(np.fft.ifft2(np.fft.fft2(Y) * np.fft.fft2(k)))[::4, ::4]
    rng = np.random.default_rng(seed)
    out = []
    for p in psnrs:
        sig = 255.0 / 10 ** (p / 20)
        out.append((blur + rng.standard_normal(blur.shape) * sig).astype(np.float32))
    return Y.astype(np.float32), u, out


def test_planted_kernel_matches_oracle_and_improves_with_psnr(cuda):
    psnrs = (10, 30, 50)
    Y, u, Xs = planted(psnrs)
    errs = []
    for p, X in zip(psnrs, Xs):
        kg, _, ki = api.estimate_kernel(torch.from_numpy(X[None].copy()).to(cuda),
                                        torch.from_numpy(Y).to(cuda), 4, 9)
        kg = to_np(kg).astype(np.float64)
        ko, _, res = oracle.estimate_kernel(X[None], Y, 4, 9)
        assert ki.status == 0
        assert rel(kg, ko) < 1e-4, p
        assert ki.iters == pytest.approx(res.iters, abs=3)
        errs.append(np.linalg.norm(kg - u) / np.linalg.norm(u))
    assert errs[0] > errs[1] > errs[2], errs
