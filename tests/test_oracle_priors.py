"""Pins of the oracle's alternative cross-channel priors (Sec. IV-D): the
generic filter machinery reproduces the LLP operator and solve already pinned
against dense and closed-form references; every prior's operator is
symmetric and positive definite; the filters act as the paper describes
(the low-pass and high-pass filters sum to the identity, the LGC filters
are the two first differences, LPP's guide is the PAN itself); guide
statistics match brute-force windows."""
import numpy as np
import pytest
from scipy import ndimage

import oracle

RNG = np.random.default_rng(321)


def _setup(H=24, W=32, c=4, R=2, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.random((2 * R + 1, 2 * R + 1))
    u /= u.sum()
    Y = rng.random((H, W)) * 255.0
    X = rng.random((H // c, W // c)) * 255.0
    return u, Y, X, c


def test_llp_through_the_generic_path_is_the_llp_operator():
    u, Y, X, c = _setup()
    st = oracle.pan_stats(Y, 1, 1.0)
    gst = oracle.prior_stats(Y, "llp", u, 1, 1.0)
    np.testing.assert_allclose(gst[0].I, st.I, rtol=0, atol=1e-9)
    np.testing.assert_allclose(gst[0].mu, st.mu, rtol=0, atol=1e-9)
    np.testing.assert_allclose(gst[0].s, st.s, rtol=1e-9)
    z = RNG.standard_normal(Y.shape)
    a = oracle.apply_z0_prior(z, u, c, oracle.prior_filters("llp", u), gst, 2e-4)
    b = oracle.apply_z0_system(z, u, c, st, 2e-4)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)
    a = oracle.apply_zstep_prior(z, u, c, oracle.prior_filters("llp", u), 2e-4)
    b = oracle.apply_zstep_system(z, u, c, 2e-4)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def test_llp_solve_through_the_generic_path():
    u, Y, X, c = _setup(seed=1)
    p = oracle.HrmsParams(tol=1e-12)
    st = oracle.pan_stats(Y, 1, 1.0)
    ref = oracle.solve_band(X, u, c, st, p)
    out = oracle.solve_band_prior(X, u, c, "llp", oracle.prior_stats(Y, "llp", u, 1, 1.0), p)
    assert np.linalg.norm(out["Z0"] - ref["Z0"]) <= 1e-8 * np.linalg.norm(ref["Z0"])
    assert np.linalg.norm(out["Z"] - ref["Z"]) <= 1e-8 * np.linalg.norm(ref["Z"])


@pytest.mark.parametrize("prior", oracle.PRIORS)
def test_prior_operators_symmetric_positive(prior):
    u, Y, X, c = _setup(seed=2)
    F = oracle.prior_filters(prior, u)
    st = oracle.prior_stats(Y, prior, u, 1, 1.0)
    z, w = RNG.standard_normal(Y.shape), RNG.standard_normal(Y.shape)
    for op in (lambda v: oracle.apply_z0_prior(v, u, c, F, st, 1e-2),
               lambda v: oracle.apply_zstep_prior(v, u, c, F, 1e-2)):
        lhs, rhs = np.vdot(op(z), w), np.vdot(z, op(w))
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
        assert np.vdot(z, op(z)) > 0


def test_filters_as_described():
    u, Y, X, c = _setup(seed=3)
    (lp,), (hp,) = oracle.prior_filters("lpf", u), oracle.prior_filters("hpf", u)
    # low-pass plus high-pass is the identity
    np.testing.assert_allclose(oracle.filt(Y, lp) + oracle.filt(Y, hp), Y, atol=1e-9)
    # the low-pass filter is the blur of the data term
    np.testing.assert_allclose(oracle.filt(Y, lp), oracle.blur_decimate(Y, u, 1), atol=1e-12)
    # lpp: the pixels themselves
    (d,) = oracle.prior_filters("lpp", u)
    np.testing.assert_allclose(oracle.filt(Y, d), Y, atol=1e-12)
    # lgc: first differences along x and y (Eq. reg2_lgc)
    h, v = oracle.prior_filters("lgc", u)
    np.testing.assert_allclose(oracle.filt(Y, h), Y - np.roll(Y, 1, axis=1), atol=1e-10)
    np.testing.assert_allclose(oracle.filt(Y, v), Y - np.roll(Y, 1, axis=0), atol=1e-10)
    # the Laplacian is the sum of the two second differences
    (L,) = oracle.prior_filters("llp", u)
    np.testing.assert_allclose(oracle.filt(Y, L), oracle.laplacian(Y), atol=1e-10)


def test_guide_stats_brute_force():
    I = RNG.standard_normal((10, 12)) * 10
    st = oracle.guide_stats(I, 1, 0.5)
    for y, x in ((0, 0), (4, 7), (9, 11)):
        win = np.array([[I[(y + i) % 10, (x + j) % 12] for j in (-1, 0, 1)] for i in (-1, 0, 1)])
        assert st.mu[y, x] == pytest.approx(win.mean(), abs=1e-12)
        assert st.s[y, x] == pytest.approx(1.0 / (win.var() + 0.5), rel=1e-12)


def test_prior_z0_solves_its_system():
    u, Y, X, c = _setup(seed=4)
    p = oracle.HrmsParams(tol=1e-12)
    for prior in ("lpf", "lgc"):
        st = oracle.prior_stats(Y, prior, u, 1, 1.0)
        out = oracle.solve_band_prior(X, u, c, prior, st, p)
        F = oracle.prior_filters(prior, u)
        b = oracle.blur_decimate_adj(X, u, c)
        res = b - oracle.apply_z0_prior(out["Z0"], u, c, F, st, p.lam)
        assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(b)
