"""Scene recipe.

Every scene is drawn from ``numpy.random.default_rng(seed)`` (PCG64) in a fixed
order, so a (config, seed) pair always yields the same arrays.

Recipe (the paper's datasets are not available; these stand in for its 4-band
and 8-band, ratio-4 workloads, Sec. IV-A):

* ground-truth HRMS, ``bands x H x W``: a background drawn as a full-canvas
  shape, then ``shapes`` ellipses or rectangles (50/50) painted in order.
  Each shape has a centre uniform on the canvas, semi-axes uniform in
  ``[4, H/4]`` and a rotation uniform in ``[0, pi)``. Its per-band intensity
  vector comes from a Gaussian copula: ``z ~ N(0, S)`` with ``S`` having unit
  diagonal and ``rho`` off the diagonal, intensity ``Phi(z)`` in ``[0, 1]``.
* texture: per band, white ``N(0, 1)`` noise, circularly Gaussian-filtered
  with ``texture_sigma`` pixels, rescaled to standard deviation
  ``texture_amp``, added. No clipping.
* PAN ``= sum_b w_b Z_b + N(0, noise^2)`` with ``w ~ Dirichlet(1, ..., 1)``.
* blur kernel ``u`` on a ``(2R+1)^2`` support, a sampled Gaussian centred at a
  sub-pixel shift, normalised to unit sum (Eq. gaussian_blur): isotropic with
  ``sigma ~ U[sigma_lo, sigma_hi]``, or anisotropic with covariance
  ``Rot(theta) diag(sx^2, sy^2) Rot(theta)^T``, ``sx, sy ~ U[sigma_lo,
  sigma_hi]``, ``theta ~ U[0, pi)``; or ("motion") the Gaussian convolved
  with a linear motion of length ``d ~ U[motion_lo, motion_hi]`` pixels
  (Appendix B): along the motion axis the difference of two Gaussian CDFs
  ``Phi(x' + d/2) - Phi(x' - d/2)``, across it a Gaussian, on coordinates
  shifted by the centre and rotated by ``theta ~ U[0, pi)``.
* LRMS ``X_b = D B(u) Z_b + N(0, noise^2)``: circular convolution
  ``(B(u) z)(y, x) = sum_{i,j} u(i, j) z(y - i, x - j)`` then keeping every
  ``ratio``-th sample at phase 0.
* all images are finally multiplied by 255: the paper states its intensities
  on the [0, 255] scale (Sec. IV-C) and its parameter values assume it.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np
from scipy.special import ndtr

SCALE = 255.0


@dataclass(frozen=True)
class SceneConfig:
    name: str
    bands: int
    H: int
    W: int
    ratio: int
    R: int                      # kernel radius, support n = 2R + 1
    shapes: int
    texture_sigma: float
    blur: str                   # "iso" or "aniso"
    sigma_lo: float
    sigma_hi: float
    shift: float                # centre offset drawn from U[-shift, shift]^2
    noise: float                # std of the PAN and LRMS noise, [0, 1] scale
    r: int = 1                  # LLP window radius
    texture_amp: float = 0.05
    rho: float = 0.8
    seed: int = 0
    motion_lo: float = 0.0      # motion length range ("motion" blur only)
    motion_hi: float = 0.0

    @property
    def n(self) -> int:
        return 2 * self.R + 1

    @property
    def h(self) -> int:
        return self.H // self.ratio

    @property
    def w(self) -> int:
        return self.W // self.ratio


CONFIGS = {
    # 4 bands, 256^2, LR 64^2, 9x9 isotropic kernel, r = 1
    "c0": SceneConfig("c0", 4, 256, 256, 4, 4, 40, 2.0, "iso", 1.0, 2.0,
                      1.0, 0.01, r=1, seed=0),
    # 8 bands, 1024^2, LR 256^2, 17x17 anisotropic kernel, r = 1 (and 2)
    "c1": SceneConfig("c1", 8, 1024, 1024, 4, 8, 200, 3.0, "aniso", 0.8, 2.5,
                      2.0, 0.005, r=1, seed=1),
    # 8 bands, 8192^2, LR 2048^2, as c1 with seed 2
    "c2": SceneConfig("c2", 8, 8192, 8192, 4, 8, 200, 3.0, "aniso", 0.8, 2.5,
                      2.0, 0.005, r=1, seed=2),
    # the paper's own setting (Sec. IV-F, Appendix B): a 29x29 support and a
    # Gaussian-times-motion blur; 4 bands, 256^2, ratio 4
    "p0": SceneConfig("p0", 4, 256, 256, 4, 14, 40, 2.0, "motion", 0.8, 1.5,
                      3.0, 0.01, r=1, seed=10, motion_lo=3.0, motion_hi=9.0),
}


def make_kernel(cfg: SceneConfig, rng: np.random.Generator) -> np.ndarray:
    """Sampled, shifted Gaussian on the (2R+1)^2 grid, unit sum (float64)."""
    R = cfg.R
    cy, cx = rng.uniform(-cfg.shift, cfg.shift, size=2)
    if cfg.blur == "motion":
        return _motion_kernel(R, cx, cy, rng.uniform(cfg.sigma_lo, cfg.sigma_hi),
                              rng.uniform(cfg.motion_lo, cfg.motion_hi),
                              rng.uniform(0.0, np.pi))
    if cfg.blur == "iso":
        s = rng.uniform(cfg.sigma_lo, cfg.sigma_hi)
        cov = np.diag([s * s, s * s])
    else:
        sx, sy = rng.uniform(cfg.sigma_lo, cfg.sigma_hi, size=2)
        th = rng.uniform(0.0, np.pi)
        rot = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        cov = rot @ np.diag([sx * sx, sy * sy]) @ rot.T
    icov = np.linalg.inv(cov)
    i, j = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    d = np.stack([j - cx, i - cy], axis=-1)          # (x, y) offsets
    q = np.einsum("...a,ab,...b->...", d, icov, d)
    u = np.exp(-0.5 * q)
    return u / u.sum()


def _motion_kernel(R: int, cx: float, cy: float, sigma: float, d: float,
                   theta: float) -> np.ndarray:
    """Gaussian (sigma) convolved with a linear motion of length d, centred
    at (cx, cy) and rotated by theta, sampled on the (2R+1)^2 grid (tap (i, j)
    at x = j, y = i), unit sum."""
    i, j = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    x, y = j - cx, i - cy
    xr = x * np.cos(theta) + y * np.sin(theta)
    yr = -x * np.sin(theta) + y * np.cos(theta)
    s = sigma * np.sqrt(2.0)
    along = ndtr((xr + 0.5 * d) / sigma) - ndtr((xr - 0.5 * d) / sigma)
    u = along * np.exp(-(yr / s) ** 2)
    return u / u.sum()


def _gauss_filter_circular(img: np.ndarray, sigma: float) -> np.ndarray:
    H, W = img.shape
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    g = np.exp(-2.0 * (np.pi * sigma) ** 2 * (fy * fy + fx * fx))
    return np.fft.irfft2(np.fft.rfft2(img) * g, s=(H, W))


def _paint_shapes(cfg: SceneConfig, rng: np.random.Generator) -> np.ndarray:
    N, H, W = cfg.bands, cfg.H, cfg.W
    cov = np.full((N, N), cfg.rho) + (1.0 - cfg.rho) * np.eye(N)
    chol = np.linalg.cholesky(cov)

    def intensity():
        return ndtr(chol @ rng.standard_normal(N))

    img = np.empty((N, H, W), dtype=np.float32)
    img[:] = intensity()[:, None, None].astype(np.float32)
    amax = max(4.0, min(H, W) / 4.0)
    for _ in range(cfg.shapes):
        kind = rng.integers(0, 2)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        ay, ax = rng.uniform(4.0, amax, size=2)
        th = rng.uniform(0.0, np.pi)
        val = intensity().astype(np.float32)
        ext = int(np.ceil(np.hypot(ay, ax))) + 1
        y0, y1 = max(0, int(cy) - ext), min(H, int(cy) + ext + 1)
        x0, x1 = max(0, int(cx) - ext), min(W, int(cx) + ext + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1, dtype=np.float64)[:, None] - cy
        xx = np.arange(x0, x1, dtype=np.float64)[None, :] - cx
        c, s = np.cos(th), np.sin(th)
        p = c * xx + s * yy
        q = -s * xx + c * yy
        if kind == 0:
            m = (p / ax) ** 2 + (q / ay) ** 2 <= 1.0
        else:
            m = (np.abs(p) <= ax) & (np.abs(q) <= ay)
        img[:, y0:y1, x0:x1][:, m] = val[:, None]
    return img


def _degrade(z: np.ndarray, u: np.ndarray, ratio: int) -> np.ndarray:
    """D B(u) z for one band, by FFT (circular convolution)."""
    H, W = z.shape
    n = u.shape[0]
    R = n // 2
    k = np.zeros((H, W))
    for i in range(-R, R + 1):
        for j in range(-R, R + 1):
            k[i % H, j % W] += u[i + R, j + R]
    full = np.fft.irfft2(np.fft.rfft2(z.astype(np.float64)) * np.fft.rfft2(k),
                         s=(H, W))
    return full[::ratio, ::ratio]


def make_scene(cfg: SceneConfig | str, seed: int | None = None) -> dict:
    """Draw one scene. Returns float32 arrays on the [0, 255] scale:
    ``hrms`` (N,H,W), ``pan`` (H,W), ``lrms`` (N,h,w), ``kernel`` (n,n) and the
    spectral weights ``weights`` (N,) used for the PAN."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    if seed is not None:
        cfg = replace(cfg, seed=seed)
    if cfg.H % cfg.ratio or cfg.W % cfg.ratio:
        raise ValueError("H and W must be multiples of the ratio")
    rng = np.random.default_rng(cfg.seed)
    u = make_kernel(cfg, rng)
    hrms = _paint_shapes(cfg, rng)
    for b in range(cfg.bands):
        t = _gauss_filter_circular(rng.standard_normal((cfg.H, cfg.W)),
                                   cfg.texture_sigma)
        t *= cfg.texture_amp / t.std()
        hrms[b] += t.astype(np.float32)
    wts = rng.dirichlet(np.ones(cfg.bands))
    pan = np.tensordot(wts, hrms.astype(np.float64), axes=1)
    pan += cfg.noise * rng.standard_normal(pan.shape)
    lrms = np.empty((cfg.bands, cfg.h, cfg.w), dtype=np.float64)
    for b in range(cfg.bands):
        lrms[b] = _degrade(hrms[b], u, cfg.ratio)
        lrms[b] += cfg.noise * rng.standard_normal(lrms[b].shape)
    return {
        "config": cfg,
        "hrms": (hrms * SCALE).astype(np.float32),
        "pan": (pan * SCALE).astype(np.float32),
        "lrms": (lrms * SCALE).astype(np.float32),
        "kernel": u.astype(np.float32),
        "weights": wts,
    }


def crop_scene(scene: dict, size: int) -> dict:
    """Top-left ``size x size`` HR crop (and the matching LR crop), to be
    treated as its own periodic scene."""
    cfg = scene["config"]
    c = cfg.ratio
    if size % c:
        raise ValueError("crop size must be a multiple of the ratio")
    out = dict(scene)
    out["config"] = replace(cfg, H=size, W=size, name=cfg.name + f"_crop{size}")
    out["hrms"] = np.ascontiguousarray(scene["hrms"][:, :size, :size])
    out["pan"] = np.ascontiguousarray(scene["pan"][:size, :size])
    out["lrms"] = np.ascontiguousarray(scene["lrms"][:, :size // c, :size // c])
    return out


def make_batch_configs(count: int = 64, seed0: int = 3000) -> list[SceneConfig]:
    """Uneven batch: side from {512, 768, 1024, 1536, 2048}, 4 or 8 bands
    (50/50), ratio 4, kernel support 9x9 ... 17x17, generated as c1."""
    rng = np.random.default_rng(seed0)
    sides = [512, 768, 1024, 1536, 2048]
    out = []
    base = CONFIGS["c1"]
    for k in range(count):
        side = int(rng.choice(sides))
        bands = int(rng.choice([4, 8]))
        R = int(rng.choice([4, 5, 6, 7, 8]))
        out.append(replace(base, name=f"c3_{k}", bands=bands, H=side, W=side,
                           R=R, seed=seed0 + k))
    return out


def _lrms_pan(cfg: SceneConfig):
    sc = make_scene(cfg)
    return sc["lrms"], sc["pan"]


def make_scenes_parallel(cfgs, workers: int | None = None) -> list:
    """(lrms, pan) of every config, generated by spawned worker processes
    (the same arrays as make_scene, in the order of cfgs)."""
    import multiprocessing as mp
    import os
    workers = max(1, min(len(cfgs), workers or os.cpu_count() or 1))
    if workers == 1:
        return [_lrms_pan(c) for c in cfgs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_lrms_pan, cfgs, chunksize=1)

