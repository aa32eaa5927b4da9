"""Training of the learned diagonal preconditioner (ps_hrms_params.precond = 2)
on the GPU, with the library's own forward, backward and Adam kernels
(include/ps_cnn.h, the weighted loss).

The diagonal network has the warm-start network's architecture and its own
parameters. Its learned part c = (net(up, pan) - up) / 255 gives the
diagonal s = max(c, 1/64) of P^{-1}. Training fits one preconditioned step
from the warm start: z_w + kappa c r_0 ~ z*, where z_w is the trained
warm-start network's output, r_0 = b - A z_w its residual in the Z0 system
of Eq. Z_ini_matting (the library's operators) and z* the band's Z0 solved
to a tight tolerance. Pixel by pixel, (kappa c r_0 - e)^2 with e = z* - z_w
is a weighted squared error of c against q = e / (kappa r_0), with weight
(kappa r_0)^2. The loss is computed as that weighted error. Details:
- kappa is the least-squares constant step over the training pixels, so that
  c is of order one;
- q is clipped to [-64, 64] (pixels with a tiny r_0, whose weight is
  negligible);
- the weights are scaled to mean one per scene.
PCG does not depend on a constant scale of s, so kappa does not reach the
solver. Data: the warm start's generator (seeded synthetic 8-band, ratio-4
scenes, kernels estimated). Usage:

    python -m paper_2103_09943_gb300.train_diag --warm weights/warm_cnn.npz --out diag.npz
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np
import torch

from . import api, ops
from .cnn import WarmStartNet

Q_CLIP = 64.0


def make_diag_dataset(n_scenes: int, size: int, seed0: int, device, warm: WarmStartNet,
                      tol: float = 1e-8, r: int = 1, eps: float = 1.0, lam: float = 2e-4):
    """[(up, pan, z_w, e, r0), ...] on the device; e = z* - z_w and
    r0 = B^T D^T X - A z_w for every band of every scene."""
    import synth
    from dataclasses import replace
    base = synth.CONFIGS["c1"]
    shapes = max(8, int(round(base.shapes * (size * size) / (base.H * base.W))))
    cfgs = [replace(base, H=size, W=size, shapes=shapes, seed=seed0 + k) for k in range(n_scenes)]
    arrays = synth.make_scenes_parallel(cfgs)
    data = []
    for cfg, (lrms, pan) in zip(cfgs, arrays):
        X = torch.from_numpy(lrms).to(device)
        Y = torch.from_numpy(pan).to(device)
        kern, _, _ = api.estimate_kernel(X, Y, cfg.ratio, cfg.R, info=False)
        hp = api.default_hrms_params(tol=tol, max_iter=20000, lam=lam, r=r, eps=eps)
        _, z0, _ = api.solve_hrms(X, Y, kern, cfg.ratio, hp, want_z0=True, info=False)
        up = ops.bicubic_up(X, cfg.ratio)
        z_w = warm.forward(up, Y)
        I, mu, s = ops.pan_stats(Y, r, eps)
        b = ops.blur_decimate_adj(X, kern, cfg.ratio)
        r0 = b - ops.apply_z0(z_w, kern, cfg.ratio, I, mu, s, r, lam)
        data.append((up, Y, z_w, z0 - z_w, r0))
    torch.cuda.synchronize()
    return data


def fit_targets(data):
    """kappa and, per scene, (up, pan, target, weight) of the weighted loss."""
    num = sum(float((e.double() * r0.double()).sum()) for _, _, _, e, r0 in data)
    den = sum(float((r0.double() ** 2).sum()) for _, _, _, e, r0 in data)
    kappa = num / den
    out = []
    for up, pan, _, e, r0 in data:
        kr = kappa * r0
        live = kr != 0
        q = torch.where(live, e / torch.where(live, kr, torch.ones_like(kr)),
                        torch.zeros_like(kr)).clamp_(-Q_CLIP, Q_CLIP)
        w = kr * kr
        w = (w / w.mean()).contiguous()
        out.append((up, pan, (up + 255.0 * q).contiguous(), w))
    return kappa, out


def train(batches, steps: int, lr: float = 1e-3, seed: int = 0, device=None, log_every: int = 0,
          net: WarmStartNet | None = None):
    """Adam with a cosine-decayed learning rate; one scene per step. The
    network starts with its last layer's bias at 1 (s = 1 everywhere, the
    plain CG) and small last-layer weights."""
    if net is None:
        net = WarmStartNet(seed=seed + 17, device=device)
        net.params[-1] = 1.0          # the last layer's bias: c = 1 before training
    rng = np.random.default_rng(seed)
    hist = []
    for it in range(steps):
        up, pan, tgt, w = batches[int(rng.integers(len(batches)))]
        loss = net.loss_grad(up, pan, tgt, weight=w)
        net.adam(lr=lr * 0.5 * (1.0 + math.cos(math.pi * it / steps)))
        hist.append(loss)
        if log_every and (it % log_every == 0 or it == steps - 1):
            print(f"step {it:5d}  loss {loss:.4e}", flush=True)
    return net, hist


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--warm", required=True, help="trained warm-start checkpoint (.npz)")
    ap.add_argument("--out", required=True, help="checkpoint (.npz) to write")
    ap.add_argument("--scenes", type=int, default=64)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--seed0", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    args = ap.parse_args(argv)
    dev = torch.device("cuda")
    warm = WarmStartNet.load(args.warm, device=dev)
    t0 = time.time()
    data = make_diag_dataset(args.scenes, args.size, args.seed0, dev, warm)
    kappa, batches = fit_targets(data)
    print(f"dataset: {len(data)} scenes of {args.size}^2 in {time.time() - t0:.1f}s; "
          f"kappa {kappa:.4e}", flush=True)
    t0 = time.time()
    net, hist = train(batches, args.steps, args.lr, device=dev, log_every=250)
    torch.cuda.synchronize()
    print(f"trained {args.steps} steps in {time.time() - t0:.1f}s; "
          f"loss {hist[0]:.4e} -> {np.mean(hist[-50:]):.4e}", flush=True)
    np.savez(args.out, params=net.params.cpu().numpy(), m=net.m.cpu().numpy(),
             v=net.v.cpu().numpy(), step=np.array(net.step), kappa=np.array(kappa))


if __name__ == "__main__":
    main()
