"""Pins of the CNN oracle (the learned warm start): the convolution against
a direct per-pixel sum and a delta image, its adjoints by the inner-product
identities, the whole backward pass by central finite differences, and Adam
against its closed form on a quadratic."""
import numpy as np
import pytest

from oracle import cnn


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 7))
    w = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    y = cnn.conv3x3(x, w, b)
    for o in range(2):
        for yy in range(5):
            for xx in range(7):
                s = b[o]
                for i in range(3):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            s += w[o, i, dy + 1, dx + 1] * x[i, (yy + dy) % 5, (xx + dx) % 7]
                assert abs(y[o, yy, xx] - s) < 1e-12


def test_conv_of_a_delta_is_the_flipped_kernel():
    # x = delta at (0, 0): out(y, x) = w[.., -y + 1, -x + 1] (torus)
    w = np.arange(9, dtype=float).reshape(1, 1, 3, 3)
    x = np.zeros((1, 6, 6))
    x[0, 0, 0] = 1.0
    y = cnn.conv3x3(x, w)[0]
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            assert y[(-dy) % 6, (-dx) % 6] == w[0, 0, dy + 1, dx + 1]


def test_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 6, 5))
    g = rng.standard_normal((3, 6, 5))
    w = rng.standard_normal((3, 4, 3, 3))
    lhs = np.sum(g * cnn.conv3x3(x, w))
    assert abs(lhs - np.sum(cnn.conv3x3_adjoint(g, w) * x)) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(cnn.conv3x3_weight_grad(x, g) * w)) < 1e-10 * abs(lhs)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = cnn.init_params(3)
    params[-1] = (params[-1][0] * 10.0, params[-1][1])     # a non-trivial last layer
    params = [(w, b + 0.01 * rng.standard_normal(b.shape)) for w, b in params]
    H = W = 8
    x = cnn.make_input(rng.random((H, W)) * 255, rng.random((H, W)) * 255)
    target = rng.random((H, W)) * 255
    z, cache = cnn.forward(params, x)
    grads = cnn.backward(params, cache, z, target)

    def L(ps):
        return cnn.loss(cnn.forward(ps, x)[0], target)

    h = 1e-6
    for l in range(cnn.n_layers()):
        w, b = params[l]
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in w.shape)
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            pp = list(params); pp[l] = (wp, b)
            pm = list(params); pm[l] = (wm, b)
            fd = (L(pp) - L(pm)) / (2 * h)
            assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1e-3, abs(fd)), (l, idx)
        j = int(rng.integers(0, b.shape[0]))
        bp, bm = b.copy(), b.copy()
        bp[j] += h
        bm[j] -= h
        pp = list(params); pp[l] = (w, bp)
        pm = list(params); pm[l] = (w, bm)
        fd = (L(pp) - L(pm)) / (2 * h)
        assert abs(fd - grads[l][1][j]) <= 1e-6 * max(1e-3, abs(fd)), (l, j)


def test_residual_output_and_zero_last_layer():
    # with the last layer zeroed the network returns its bicubic input
    rng = np.random.default_rng(4)
    params = cnn.init_params(5)
    params[-1] = (np.zeros_like(params[-1][0]), np.zeros(1))
    up = rng.random((6, 6)) * 255
    z, _ = cnn.forward(params, cnn.make_input(up, rng.random((6, 6)) * 255))
    np.testing.assert_allclose(z, up, rtol=0, atol=1e-12)


def test_adam_first_steps_closed_form():
    # first Adam step moves every coordinate by lr * sign(g) (bias-corrected
    # m / sqrt(v) = g / |g|), up to eps
    p = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    g = [(np.array([[0.3, -4.0]]), np.array([-1e-3]))]
    st = {}
    out = cnn.adam_step(p, g, st, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(out[0][0], [[0.99, -1.99]], atol=1e-9)
    np.testing.assert_allclose(out[0][1], [0.51], atol=1e-9)
    assert st["t"] == 1
