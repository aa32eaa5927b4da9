"""Dense matrices assembled directly from the paper's definitions, for tiny
tori. Written independently of the oracle (different formulas, explicit
enumeration of windows and taps), so that agreement pins the oracle.
"""
from __future__ import annotations

import numpy as np


def conv_matrix(u: np.ndarray, H: int, W: int) -> np.ndarray:
    """B(u): (B z)(y, x) = sum_{i,j} u(i, j) z(y - i, x - j), circular."""
    n = u.shape[0]
    R = n // 2
    B = np.zeros((H * W, H * W))
    for y in range(H):
        for x in range(W):
            for i in range(-R, R + 1):
                for j in range(-R, R + 1):
                    B[y * W + x, ((y - i) % H) * W + (x - j) % W] += u[i + R, j + R]
    return B


def decimation_matrix(H: int, W: int, c: int) -> np.ndarray:
    """D: keeps the samples (c k, c l)."""
    h, w = H // c, W // c
    D = np.zeros((h * w, H * W))
    for k in range(h):
        for l in range(w):
            D[k * w + l, (c * k) * W + c * l] = 1.0
    return D


def laplacian_matrix(H: int, W: int) -> np.ndarray:
    S = {(0, 0): 4.0, (-1, 0): -1.0, (1, 0): -1.0, (0, -1): -1.0, (0, 1): -1.0}
    L = np.zeros((H * W, H * W))
    for y in range(H):
        for x in range(W):
            for (dy, dx), v in S.items():
                L[y * W + x, ((y + dy) % H) * W + (x + dx) % W] += v
    return L


def windows(H: int, W: int, r: int):
    """Flat pixel indices of every (2r+1)^2 torus window, one per centre."""
    out = []
    for y in range(H):
        for x in range(W):
            out.append([((y + dy) % H) * W + (x + dx) % W
                        for dy in range(-r, r + 1) for dx in range(-r, r + 1)])
    return out


def matting_matrix(I: np.ndarray, r: int, eps: float) -> np.ndarray:
    """Eq. matting_matrix with sigma_k^2 + eps in the denominator:
    M_mn = sum_{k : m, n in w_k} [delta_mn - (1/|w|)(1 + (I_m - mu_k)(I_n - mu_k)
           / (sigma_k^2 + eps))]."""
    H, W = I.shape
    flat = I.ravel()
    M = np.zeros((H * W, H * W))
    for win in windows(H, W, r):
        vals = flat[win]
        mu = vals.mean()
        var = vals.var()
        nw = len(win)
        for a, m in enumerate(win):
            for b, nn in enumerate(win):
                M[m, nn] += (1.0 if m == nn else 0.0) - (1.0 / nw) * (
                    1.0 + (vals[a] - mu) * (vals[b] - mu) / (var + eps))
    return M


def grad_matrices(n: int):
    """Circular forward differences on the n x n kernel grid, as matrices."""
    N = n * n
    Dh = np.zeros((N, N))
    Dv = np.zeros((N, N))
    for i in range(n):
        for j in range(n):
            m = i * n + j
            Dh[m, i * n + (j + 1) % n] += 1.0
            Dh[m, m] -= 1.0
            Dv[m, ((i + 1) % n) * n + j] += 1.0
            Dv[m, m] -= 1.0
    return Dh, Dv


def fft_conv(z: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Circular convolution by numpy's FFT."""
    H, W = z.shape
    R = u.shape[0] // 2
    k = np.zeros((H, W))
    for i in range(-R, R + 1):
        for j in range(-R, R + 1):
            k[i % H, j % W] += u[i + R, j + R]
    return np.real(np.fft.ifft2(np.fft.fft2(z) * np.fft.fft2(k)))
