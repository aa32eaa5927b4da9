"""Checks of the input generator's motion-blur kernel (Appendix B): with no
motion it is the sampled isotropic Gaussian; its spread along the motion
axis is that of a Gaussian plus a uniform segment (sigma^2 + d^2 / 12)."""
import numpy as np

from synth.scenes import _motion_kernel


def test_no_motion_is_the_isotropic_gaussian():
    R, s, cx, cy = 6, 1.3, 0.4, -0.7
    u = _motion_kernel(R, cx, cy, s, 1e-6, 0.9)
    i, j = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    g = np.exp(-((j - cx) ** 2 + (i - cy) ** 2) / (2 * s * s))
    # far tails: the difference of two CDFs near 1 loses everything below 1e-16
    np.testing.assert_allclose(u, g / g.sum(), rtol=1e-5, atol=1e-10)


def test_second_moments_along_and_across_the_motion():
    R, s, d, th = 20, 1.0, 9.0, 0.6
    u = _motion_kernel(R, 0.0, 0.0, s, d, th)
    i, j = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    a = j * np.cos(th) + i * np.sin(th)          # along the motion
    b = -j * np.sin(th) + i * np.cos(th)         # across it
    assert abs(np.sum(u * a)) < 1e-9 and abs(np.sum(u * b)) < 1e-9
    # sampling a smooth density on the unit grid keeps its moments to ~1e-3
    assert abs(np.sum(u * a * a) - (s * s + d * d / 12.0)) < 1e-2
    assert abs(np.sum(u * b * b) - s * s) < 1e-2
    assert abs(np.sum(u * a * b)) < 1e-2
