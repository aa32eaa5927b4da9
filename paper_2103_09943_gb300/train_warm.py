"""Training of the learned warm start on the GPU, with the library's own
forward, backward and Adam kernels (include/ps_cnn.h).

Data: seeded synthetic scenes from the 8-band, ratio-4 generator (17 x 17
anisotropic kernels) at a reduced size; for each scene the kernel is estimated
(Algorithm 1) and every band's Z0 (Eq. Z_ini_matting) is solved to a tight
tolerance by the library: the targets are the method's own solutions. The
network's inputs are the bicubic upsampling of the LRMS band and the PAN.
Batches are whole (periodic) scenes, so the network's circular padding sees
no crop seams. Usage:

    python -m paper_2103_09943_gb300.train_warm --out warm.npz
"""
from __future__ import annotations

import argparse
import math
import time
from dataclasses import replace

import numpy as np
import torch

from . import api, ops
from .cnn import WarmStartNet


def make_dataset(n_scenes: int, size: int, seed0: int, device, tol: float = 1e-8):
    """[(up (N,H,W), pan (H,W), z0 (N,H,W)), ...] on the device."""
    import synth
    base = synth.CONFIGS["c1"]
    shapes = max(8, int(round(base.shapes * (size * size) / (base.H * base.W))))
    cfgs = [replace(base, H=size, W=size, shapes=shapes, seed=seed0 + k) for k in range(n_scenes)]
    arrays = synth.make_scenes_parallel(cfgs)   # host cores, spawned workers
    data = []
    for cfg, (lrms, pan) in zip(cfgs, arrays):
        X = torch.from_numpy(lrms).to(device)
        Y = torch.from_numpy(pan).to(device)
        kern, _, _ = api.estimate_kernel(X, Y, cfg.ratio, cfg.R, info=False)
        hp = api.default_hrms_params(tol=tol, max_iter=20000)
        _, z0, _ = api.solve_hrms(X, Y, kern, cfg.ratio, hp, want_z0=True, info=False)
        data.append((ops.bicubic_up(X, cfg.ratio), Y, z0))
    torch.cuda.synchronize()
    return data


def train(data, steps: int, lr: float = 2e-3, seed: int = 0, device=None, log_every: int = 0,
          net: WarmStartNet | None = None):
    """Adam with a cosine-decayed learning rate; one scene (all its bands)
    per step, scenes in a seeded random order."""
    net = net or WarmStartNet(seed=seed, device=device)
    rng = np.random.default_rng(seed)
    hist = []
    for it in range(steps):
        up, pan, z0 = data[int(rng.integers(len(data)))]
        loss = net.loss_grad(up, pan, z0)
        net.adam(lr=lr * 0.5 * (1.0 + math.cos(math.pi * it / steps)))
        hist.append(loss)
        if log_every and (it % log_every == 0 or it == steps - 1):
            print(f"step {it:5d}  loss {loss:.4e}", flush=True)
    return net, hist


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True, help="checkpoint (.npz) to write")
    ap.add_argument("--scenes", type=int, default=96)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--resume", default=None, help="checkpoint to continue from")
    args = ap.parse_args(argv)
    dev = torch.device("cuda")
    t0 = time.time()
    data = make_dataset(args.scenes, args.size, args.seed0, dev)
    print(f"dataset: {len(data)} scenes of {args.size}^2 in {time.time() - t0:.1f}s", flush=True)
    net = WarmStartNet.load(args.resume, device=dev) if args.resume else None
    t0 = time.time()
    net, hist = train(data, args.steps, args.lr, device=dev, log_every=250, net=net)
    torch.cuda.synchronize()
    print(f"trained {args.steps} steps in {time.time() - t0:.1f}s; "
          f"loss {hist[0]:.4e} -> {np.mean(hist[-50:]):.4e}", flush=True)
    net.save(args.out)


if __name__ == "__main__":
    main()
