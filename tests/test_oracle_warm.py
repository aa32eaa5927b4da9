"""Pins of the oracle's bicubic warm start (Keys cubic convolution, a = -0.5,
phase-0 alignment, circular boundary): interpolation, partition of unity,
exact reproduction of polynomials up to degree 2 away from the wrap, and the
kernel's closed-form values."""
import numpy as np

import oracle


def test_keys_kernel_values():
    W = oracle.fbmp.keys_cubic
    assert W(0.0) == 1.0 and W(1.0) == 0.0 and W(2.0) == 0.0 and W(2.5) == 0.0
    # W(1/2) = (a+2)/8 - (a+3)/4 + 1 = 0.5625 and W(3/2) = -0.0625 at a = -1/2
    assert abs(W(0.5) - 0.5625) < 1e-15 and abs(W(1.5) + 0.0625) < 1e-15
    # the four weights of any phase sum to one
    for t in np.linspace(0, 1, 7):
        assert abs(W(t - np.arange(-1, 3)).sum() - 1.0) < 1e-14


def test_interpolates_lr_samples_and_constants():
    rng = np.random.default_rng(0)
    X = rng.random((2, 9, 12))
    for c in (2, 3, 4):
        U = oracle.bicubic_up(X, c)
        assert U.shape == (2, 9 * c, 12 * c)
        np.testing.assert_allclose(U[:, ::c, ::c], X, rtol=0, atol=1e-14)
    np.testing.assert_allclose(oracle.bicubic_up(np.full((6, 8), 3.25), 4), 3.25, atol=1e-14)


def test_reproduces_quadratics_away_from_the_wrap():
    h, w, c = 16, 16, 4
    ky, kx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    f = lambda y, x: 0.3 * y * y - 0.7 * x * y + 2.0 * x + 1.0
    U = oracle.bicubic_up(f(ky, kx).astype(float), c)
    Y, X = np.meshgrid(np.arange(h * c) / c, np.arange(w * c) / c, indexing="ij")
    inner = (slice(2 * c, (h - 3) * c), slice(2 * c, (w - 3) * c))
    np.testing.assert_allclose(U[inner], f(Y, X)[inner], rtol=0, atol=1e-10)


def test_circular_boundary():
    # a unit impulse at LR (0, 0) spreads to HR rows/cols on both sides of the wrap
    X = np.zeros((8, 8))
    X[0, 0] = 1.0
    U = oracle.bicubic_up(X, 2)
    W = oracle.fbmp.keys_cubic
    assert abs(U[-1, 0] - W(0.5)) < 1e-15        # HR row -1 = LR coordinate -1/2
    assert abs(U[-3, -3] - W(1.5) ** 2) < 1e-15  # LR (-3/2, -3/2)
