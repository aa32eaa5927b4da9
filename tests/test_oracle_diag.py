"""Pins of the oracle's learned diagonal preconditioner (an extension of the
Z0 CG of Eq. Z_ini_matting: the paper runs plain CG).

Diagonal PCG is checked against a LAPACK solve of the dense Z0 system,
iterate by iterate against plain CG on the symmetrically scaled dense system
S^1/2 A S^1/2 (the textbook identity behind a diagonal preconditioner), and
against the oracle's plain CG when s is constant. The network side: the
weighted loss by finite differences and its weight-1 special case, and the
training target by the one-step error it stands for."""
import numpy as np
import pytest

import oracle
import synth
from oracle import cnn
from tests.test_oracle_operators import _dense_A, kern


def _tiny(seed=11):
    H, W, c, R, r, eps, lam = 32, 32, 4, 3, 1, 1.0, 2e-4
    rng = np.random.default_rng(seed)
    u = kern(R, rng)
    Y = rng.random((H, W)) * 255
    X = rng.random((H // c, W // c)) * 255
    A, B, D, L = _dense_A(H, W, c, u, Y, r, eps, lam)
    b = (B.T @ D.T @ X.ravel()).reshape(H, W)
    st = oracle.pan_stats(Y, r, eps)
    s = np.exp(rng.uniform(-1.5, 1.5, (H, W)))       # positive, spread over e^3
    return dict(H=H, W=W, c=c, u=u, lam=lam, A=A, b=b, st=st, s=s, rng=rng)


def test_diag_pcg_matches_dense_solve():
    t = _tiny()
    ref = np.linalg.solve(t["A"], t["b"].ravel()).reshape(t["H"], t["W"])
    z, it, rel = oracle.pcg_diag_solve(t["b"], t["u"], t["c"], t["lam"], t["st"], t["s"],
                                       tol=1e-12)
    assert rel <= 1e-12
    assert oracle.rel_l2(z, ref) < 1e-9


@pytest.mark.parametrize("k", [1, 2, 7, 20])
def test_diag_pcg_is_cg_on_the_scaled_system(k):
    # PCG with P^{-1} = S = diag(s) from x0 produces x_k = S^1/2 y_k, y_k the
    # plain-CG iterates on (S^1/2 A S^1/2) y = S^1/2 b from y0 = S^-1/2 x0
    t = _tiny(13)
    A, b, s = t["A"], t["b"].ravel(), t["s"].ravel()
    x0 = t["rng"].standard_normal(b.size) * 10
    h = np.sqrt(s)
    Ah = h[:, None] * A * h[None, :]
    bh = h * b
    y = x0 / h
    r = bh - Ah @ y
    p = r.copy()
    rr = r @ r
    for _ in range(k):
        q = Ah @ p
        a = rr / (p @ q)
        y = y + a * p
        r = r - a * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
    x, it, _ = oracle.pcg_diag_solve(t["b"], t["u"], t["c"], t["lam"], t["st"], t["s"],
                                     x0=x0.reshape(t["H"], t["W"]), tol=0.0, max_iter=k)
    assert it == k
    assert oracle.rel_l2(x.ravel(), h * y) < 1e-10


def test_constant_diagonal_is_plain_cg():
    # P^{-1} = kappa I gives plain CG's iterates (scale invariance): same
    # count, same solution as the oracle's C routine
    sc = synth.crop_scene(synth.make_scene(synth.CONFIGS["c0"]), 64)
    c, lam = 4, 2e-4
    u = sc["kernel"].astype(np.float64)
    st = oracle.pan_stats(sc["pan"], 1, 1.0)
    b = oracle.blur_decimate_adj(sc["lrms"][0], u, c)
    z_cg, it_cg, _ = oracle.cg_solve(0, b, u, c, lam, st, tol=1e-9)
    z_d, it_d, rel = oracle.pcg_diag_solve(b, u, c, lam, st, np.full(b.shape, 37.5), tol=1e-9)
    assert rel <= 1e-9
    assert abs(it_d - it_cg) <= 1
    assert oracle.rel_l2(z_d, z_cg) < 1e-7


def test_diag_pcg_rejects_nonpositive_diagonal():
    t = _tiny()
    s = t["s"].copy()
    s[3, 4] = 0.0
    with pytest.raises(ValueError):
        oracle.pcg_diag_solve(t["b"], t["u"], t["c"], t["lam"], t["st"], s)


def test_weighted_loss_gradient_by_finite_differences():
    rng = np.random.default_rng(21)
    params = cnn.init_params(7)
    params[-1] = (params[-1][0] * 10.0, params[-1][1])
    H = W = 8
    x = cnn.make_input(rng.random((H, W)) * 255, rng.random((H, W)) * 255)
    target = rng.random((H, W)) * 255
    weight = rng.random((H, W)) * 3.0
    z, cache = cnn.forward(params, x)
    grads = cnn.backward(params, cache, z, target, weight=weight)

    def L(ps):
        return cnn.loss(cnn.forward(ps, x)[0], target, weight)

    h = 1e-6
    for l in range(cnn.n_layers()):
        w, b = params[l]
        for _ in range(3):
            idx = tuple(rng.integers(0, n) for n in w.shape)
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            pp = list(params); pp[l] = (wp, b)
            pm = list(params); pm[l] = (wm, b)
            fd = (L(pp) - L(pm)) / (2 * h)
            assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1e-3, abs(fd)), (l, idx)
    # weight 1 is the plain loss, gradient for gradient
    g1 = cnn.backward(params, cache, z, target, weight=np.ones((H, W)))
    g0 = cnn.backward(params, cache, z, target)
    for (a, b), (c, d) in zip(g1, g0):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(b, d)
    assert cnn.loss(z, target, np.ones((H, W))) == cnn.loss(z, target)


def test_diag_fit_is_the_one_step_error():
    # with z = s (x_0 + c), the weighted loss of diag_fit's (target, weight)
    # is the mean one-step error (kappa c r_0 - e)^2, for any c
    rng = np.random.default_rng(23)
    H = W = 12
    up = rng.random((H, W)) * 255
    z_w = up + rng.standard_normal((H, W)) * 5
    z_star = z_w + rng.standard_normal((H, W)) * 2
    r0 = rng.standard_normal((H, W)) * 0.3
    r0[2, 3] = 0.0
    kappa = 4.5
    tgt, wt = cnn.diag_fit(up, z_w, z_star, r0, kappa)
    for _ in range(3):
        c = rng.standard_normal((H, W))
        z = up + cnn.SCALE * c
        one_step = np.mean((kappa * c * r0 - (z_star - z_w)) ** 2)
        # the r_0 = 0 pixel contributes e^2 to the one-step error, 0 to the loss
        e0 = (z_star - z_w)[2, 3] ** 2 / (H * W)
        assert abs(cnn.loss(z, tgt, wt) - (one_step - e0)) < 1e-10 * one_step
    # the head: floor where the learned part is small, negative or not finite
    c = np.array([[2.0, -1.0], [1e-4, np.nan]])
    s = cnn.diag_head(up[:2, :2] + cnn.SCALE * c, up[:2, :2])
    np.testing.assert_allclose(s, [[2.0, cnn.DIAG_FLOOR], [cnn.DIAG_FLOOR, cnn.DIAG_FLOOR]],
                               rtol=1e-12)


@pytest.mark.parametrize("H,W,c,R,r,lam", [(16, 16, 4, 2, 1, 2e-2), (12, 20, 2, 3, 1, 5e-3),
                                           (18, 12, 3, 2, 2, 1e-1)])
def test_jacobi_diag_is_the_dense_operators_diagonal(H, W, c, R, r, lam):
    # diag(B^T D^T D B + lam L^T M L) assembled entry by entry (dense matrices
    # from the definitions), against the oracle's per-pixel formula; a
    # non-square torus, ratios 2-4, window radius 1 and 2
    rng = np.random.default_rng(H * W + c + R + r)
    u = kern(R, rng)
    Y = rng.random((H, W)) * 255
    A, *_ = _dense_A(H, W, c, u, Y, r, 1.0, lam)
    st = oracle.pan_stats(Y, r, 1.0)
    d = oracle.jacobi_diag(u, c, st, lam)
    np.testing.assert_allclose(d.ravel(), np.diag(A), rtol=1e-11, atol=1e-12)
    assert d.min() > 0


def test_jacobi_pcg_reaches_the_dense_solution():
    # the Jacobi preconditioner, s = 1 / diag(A), in the oracle's diagonal PCG
    t = _tiny(13)
    s = 1.0 / oracle.jacobi_diag(t["u"], t["c"], t["st"], t["lam"])
    assert np.allclose(s.ravel(), 1.0 / np.diag(t["A"]), rtol=1e-11)
    ref = np.linalg.solve(t["A"], t["b"].ravel()).reshape(t["H"], t["W"])
    z, it, rel = oracle.pcg_diag_solve(t["b"], t["u"], t["c"], t["lam"], t["st"], s, tol=1e-12)
    assert oracle.rel_l2(z, ref) < 1e-9
