"""Helpers shared by the GPU parity tests."""
import numpy as np
import torch


def to_dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)


def to_np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rand_kernel(R, rng):
    u = rng.random((2 * R + 1, 2 * R + 1)) + 0.05
    return u / u.sum()
