"""Pins of the oracle's kernel estimate (Algorithm 1) and of Algorithm 2's
block-coordinate step (CPU only)."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from oracle import fbmp
from tests import dense_ref


def _project_bisect(v, iters=200):
    # tau solves sum max(v + tau, 0) = 1 (monotone in tau): bisection.
    lo, hi = -v.max() - 1.0, -v.min() + 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if np.maximum(v + mid, 0).sum() > 1.0:
            hi = mid
        else:
            lo = mid
    return np.maximum(v + 0.5 * (lo + hi), 0)


def _project_brute(v):
    # Every support S: x_S = v_S + tau, tau = (1 - sum v_S)/|S|; keep the
    # feasible candidate closest to v.
    best, bd = None, np.inf
    n = v.size
    for k in range(1, n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            tau = (1.0 - v[S].sum()) / len(S)
            x = np.zeros(n)
            x[S] = v[S] + tau
            if x.min() < -1e-15:
                continue
            d = np.sum((x - v) ** 2)
            if d < bd:
                best, bd = x, d
    return best


@pytest.mark.parametrize("seed", range(6))
def test_simplex_projection(seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(25) * (0.1 + seed)
    if seed == 3:
        v[:5] = v[0]                      # ties
    x = oracle.simplex_project(v)
    assert x.min() >= 0 and x.sum() == pytest.approx(1.0, abs=1e-13)
    np.testing.assert_allclose(x, _project_bisect(v), atol=1e-12)
    # KKT: x - v = tau on the support, and x_i = 0 only where v_i + tau <= 0.
    sup = x > 0
    tau = np.mean((x - v)[sup])
    np.testing.assert_allclose((x - v)[sup], tau, atol=1e-12)
    assert np.all(v[~sup] + tau <= 1e-12)
    w = v[:9]
    np.testing.assert_allclose(oracle.simplex_project(w), _project_brute(w), atol=1e-12)


def test_shrink2_is_the_prox():
    # shrink2(e, t) minimises t||x|| + 1/2||x - e||^2 per row (Eq. x_update):
    # the optimality condition x - e + t x/||x|| = 0 for ||e|| > t, else x = 0.
    rng = np.random.default_rng(0)
    e = rng.standard_normal((4, 50))
    t = 1.2
    x = fbmp.shrink2(e, t)
    nx = np.linalg.norm(x, axis=0)
    ne = np.linalg.norm(e, axis=0)
    big = ne > t
    np.testing.assert_allclose(nx[big], ne[big] - t, atol=1e-13)
    g = x[:, big] - e[:, big] + t * x[:, big] / nx[big]
    assert np.max(np.abs(g)) < 1e-12
    assert np.all(x[:, ~big] == 0)


@pytest.mark.parametrize("n", [5, 7])
def test_up_solve_satisfies_spatial_normal_equations(n):
    # The Fourier/Cramer solution of Eq. u_p_solution must make the gradient
    # of the {u, p} objective (with the mu3 coupling) vanish. The gradient is
    # evaluated with dense difference matrices built independently, and the
    # solution is also compared with a dense solve of the block system.
    rng = np.random.default_rng(n)
    kp = oracle.KernelParams(alpha1=0.7, alpha2=0.05, mu1=3.0, mu2=5.0, mu3=2.0)
    x = rng.standard_normal((2, n, n))
    y = rng.standard_normal((4, n, n))
    y[2] = y[1]
    L1 = rng.standard_normal((2, n, n))
    L2 = rng.standard_normal((4, n, n))
    L2[2] = L2[1]
    L3 = rng.standard_normal((n, n))
    z = rng.standard_normal((n, n))
    u, p1, p2 = oracle.up_solve(x, y, z, L1, L2, L3, kp)
    Dh, Dv = dense_ref.grad_matrices(n)
    a1, a2 = kp.alpha1 * kp.mu1, kp.alpha2 * kp.mu2
    f = lambda a: a.ravel()
    U, P1, P2 = f(u), f(p1), f(p2)
    e1 = Dh @ U - P1 - f(x[0] - L1[0])
    e2 = Dv @ U - P2 - f(x[1] - L1[1])
    m = 0.5 * (Dv @ P1 + Dh @ P2)
    g1 = Dh @ P1 - f(y[0] - L2[0])
    g2 = m - f(y[1] - L2[1])
    g3 = m - f(y[2] - L2[2])
    g4 = Dv @ P2 - f(y[3] - L2[3])
    e3 = U - f(z - L3)
    gu = a1 * (Dh.T @ e1 + Dv.T @ e2) + kp.mu3 * e3
    gp1 = -a1 * e1 + a2 * (Dh.T @ g1 + 0.5 * Dv.T @ g2 + 0.5 * Dv.T @ g3)
    gp2 = -a1 * e2 + a2 * (Dv.T @ g4 + 0.5 * Dh.T @ g2 + 0.5 * Dh.T @ g3)
    scale = np.max(np.abs(np.concatenate([U, P1, P2]))) * (a1 + a2 + kp.mu3)
    for g in (gu, gp1, gp2):
        assert np.max(np.abs(g)) < 1e-11 * scale
    # Dense block system of Eq. block_toeplitz (+ mu3 I in d1).
    N = n * n
    I = np.eye(N)
    d1 = a1 * (Dh.T @ Dh + Dv.T @ Dv) + kp.mu3 * I
    d2 = a1 * I + a2 * Dh.T @ Dh + 0.5 * a2 * Dv.T @ Dv
    d3 = a1 * I + a2 * Dv.T @ Dv + 0.5 * a2 * Dh.T @ Dh
    d4, d5, d6 = -a1 * Dh, -a1 * Dv, 0.5 * a2 * Dh.T @ Dv
    K = np.block([[d1, d4.T, d5.T], [d4, d2, d6.T], [d5, d6, d3]])
    B1 = a1 * (Dh.T @ f(x[0] - L1[0]) + Dv.T @ f(x[1] - L1[1])) + kp.mu3 * f(z - L3)
    B2 = a1 * f(L1[0] - x[0]) + a2 * (Dh.T @ f(y[0] - L2[0]) + Dv.T @ f(y[1] - L2[1]))
    B3 = a1 * f(L1[1] - x[1]) + a2 * (Dv.T @ f(y[3] - L2[3]) + Dh.T @ f(y[1] - L2[1]))
    sol = np.linalg.solve(K, np.concatenate([B1, B2, B3]))
    np.testing.assert_allclose(np.concatenate([U, P1, P2]), sol, atol=1e-11)


def _noiseless_scene(H=128, R=3, c=4, blur=True, seed=21):
    cfg = synth.CONFIGS["c0"]
    from dataclasses import replace
    cfg = replace(cfg, H=H, W=H, R=R, noise=0.0, seed=seed)
    sc = synth.make_scene(cfg)
    Z = sc["hrms"].astype(np.float64)
    w = sc["weights"]
    Y = np.tensordot(w, Z, axes=1)          # exact PAN, no noise
    if blur:
        u = sc["kernel"].astype(np.float64)
        u /= u.sum()
        X = np.stack([dense_ref.fft_conv(Z[b], u)[::c, ::c] for b in range(Z.shape[0])])
    else:
        u = None
        X = Z[:, ::c, ::c].copy()
    return Z, Y, X, u, w


def test_omega_exact_recovery_without_blur():
    # With no blur, no noise, l = 0 (u1 = u2 = identity) and lambda_omega = 0,
    # D Y = sum_b w_b X_b exactly, so Eq. objective3 recovers w.
    Z, Y, X, _, w = _noiseless_scene(blur=False)
    om = oracle.estimate_omega(X, Y, 4, 0, 0.0)
    np.testing.assert_allclose(om, w, rtol=1e-9)


def test_omega_over_a_band_subset():
    # X' of Eq. objective1: a PAN made of bands {0, 2} only. Over that subset
    # the weights are recovered exactly (no blur, no noise, l = 0); the
    # kernel estimate restricted to it combines only those bands, and with
    # the weights given it equals the estimate from f = X' omega by hand.
    Z, _, X, u, w = _noiseless_scene(blur=True, H=64)
    bands = [0, 2]
    wt = np.array([0.6, 0.4])
    Y = np.tensordot(wt, Z[bands], axes=1)
    Xn = Z[:, ::4, ::4]                  # unblurred LRMS for the exact recovery
    np.testing.assert_allclose(oracle.estimate_omega(Xn, Y, 4, 0, 0.0, bands=bands), wt,
                               rtol=1e-9)
    # all four bands: the least-squares fit still finds the PAN's mix
    om4 = oracle.estimate_omega(Xn, Y, 4, 0, 0.0)
    np.testing.assert_allclose(om4[bands], wt, rtol=1e-6)
    np.testing.assert_allclose(om4[[1, 3]], 0.0, atol=1e-6)
    kp = oracle.KernelParams(t_max=200)
    k_sub, om_sub, _ = oracle.estimate_kernel(X, Y, 4, 3, kp, omega=wt, bands=bands)
    f = np.tensordot(wt, X[bands], axes=1)
    EtE, Etf = oracle.kernel_normal_eq(Y, f, 4, 3)
    np.testing.assert_allclose(k_sub, oracle.admm(EtE, Etf, 3, kp).kernel, atol=1e-14)


def test_omega_regularised_matches_lstsq():
    from scipy import ndimage
    Z, Y, X, _, w = _noiseless_scene(H=64)
    c, l, lam = 4, 2, 1e6
    om = oracle.estimate_omega(X, Y, c, l, lam)
    A = np.stack([ndimage.uniform_filter(X[k], 2 * l + 1, mode="wrap").ravel()
                  for k in range(X.shape[0])], axis=1)
    b = ndimage.uniform_filter(Y, 2 * c * l + 1, mode="wrap")[::c, ::c].ravel()
    G = np.diff(np.eye(X.shape[0]), axis=0)
    ref, *_ = np.linalg.lstsq(np.vstack([A, np.sqrt(lam) * G]),
                              np.concatenate([b, np.zeros(G.shape[0])]), rcond=None)
    np.testing.assert_allclose(om, ref, rtol=1e-8)


def test_planted_kernel_recovery():
    # Noiseless data blurred by a planted kernel, omega given: the ADMM of
    # Algorithm 1 with weak regularisation recovers it (Eq. relative_error_kernel
    # below 1 %), and the z = u splitting residual vanishes.
    Z, Y, X, u_true, w = _noiseless_scene(H=128, R=3)
    kp = oracle.KernelParams(alpha1=1e-6, alpha2=1e-6, t_max=20000, th=1e-9)
    k, om, res = oracle.estimate_kernel(X, Y, 4, 3, kp, omega=w)
    assert oracle.kernel_error_pct(k, u_true) < 1.0
    assert res.primal["z"] < 1e-6


def test_admm_limit_without_regulariser_is_the_constrained_minimiser():
    # Algorithm 1 projects the unconstrained z solve onto the simplex
    # (Eq. z_solution, then the projection). With alpha1, alpha2 -> 0 this is
    # a proximal-point iteration whose fixed point is the simplex-constrained
    # least-squares minimiser exactly when E^T E is a multiple of I; then the
    # minimiser is P_S(E^T f / kappa), computed here by bisection.
    rng = np.random.default_rng(2)
    R = 2
    nn = (2 * R + 1) ** 2
    kappa = 100.0
    g = rng.standard_normal(nn) * 30 + 4
    kp = oracle.KernelParams(alpha1=1e-12, alpha2=1e-12, t_max=5000, th=1e-13)
    res = oracle.admm(kappa * np.eye(nn), g, R, kp)
    np.testing.assert_allclose(res.kernel.ravel(), _project_bisect(g / kappa),
                               atol=1e-9)


def _pansharp_objective(Z, X, Y, u, c, lam, eps, r, A, C):
    """Eq. pansharp for one band, evaluated by explicit window sums."""
    LZ = oracle.laplacian(Z)
    I = oracle.laplacian(Y)
    H, W = Z.shape
    data = 0.5 * np.sum((dense_ref.fft_conv(Z, u)[::c, ::c] - X) ** 2)
    prior = 0.0
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            # window centred at j contains k = j + (dy, dx)
            LZk = np.roll(np.roll(LZ, -dy, 0), -dx, 1)
            Ik = np.roll(np.roll(I, -dy, 0), -dx, 1)
            prior += np.sum((LZk - A * Ik - C) ** 2 + eps * A ** 2)
    return data + 0.5 * lam * prior


def test_block_step_with_exact_weight_does_not_increase_objective():
    # Algorithm 2's one block-coordinate pass: (A, C) from the guided filter
    # are the exact minimisers given Z0, and the Z step with weight lam|w| is
    # the exact minimiser given (A, C); so Eq. pansharp cannot increase.
    sc = synth.make_scene("c0")
    c, R = 4, 4
    Y = sc["pan"][:64, :64].astype(np.float64)
    X = sc["lrms"][0, :16, :16].astype(np.float64)
    u = sc["kernel"].astype(np.float64)
    hp = oracle.HrmsParams(exact_weight=True, tol=1e-12)
    st = oracle.pan_stats(Y, hp.r, hp.eps)
    out = oracle.solve_band(X, u, c, st, hp)
    q = oracle.laplacian(out["Z0"])
    a = np.empty_like(q)
    Cc = np.empty_like(q)
    nw = (2 * hp.r + 1) ** 2
    box = lambda t: sum(np.roll(np.roll(t, -dy, 0), -dx, 1)
                        for dy in range(-1, 2) for dx in range(-1, 2)) / nw
    a = (box(st.I * q) - st.mu * box(q)) * st.s
    Cc = box(q) - a * st.mu
    f0 = _pansharp_objective(out["Z0"], X, Y, u, c, hp.lam, hp.eps, hp.r, a, Cc)
    f1 = _pansharp_objective(out["Z"], X, Y, u, c, hp.lam, hp.eps, hp.r, a, Cc)
    assert f1 <= f0 * (1 + 1e-12)
    # and perturbing Z away from the Z-step solution increases it
    rng = np.random.default_rng(0)
    f2 = _pansharp_objective(out["Z"] + 0.5 * rng.standard_normal(out["Z"].shape),
                             X, Y, u, c, hp.lam, hp.eps, hp.r, a, Cc)
    assert f2 > f1
