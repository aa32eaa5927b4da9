"""Pins of the oracle's image-domain operators (CPU only).

Each check compares the oracle with something other than itself: numpy's
FFT or scipy's filters on special cases, dense matrices assembled directly
from the paper's definitions, adjoint identities, brute force on tiny tori.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
from tests import dense_ref

RNG = np.random.default_rng(1234)


def rand(*shape):
    return RNG.standard_normal(shape)


def kern(R, rng=RNG):
    u = rng.random((2 * R + 1, 2 * R + 1))
    return u / u.sum()


@pytest.mark.parametrize("H,W,c,R", [(24, 32, 4, 3), (20, 28, 4, 4),
                                     (18, 12, 2, 2), (9, 15, 3, 1)])
def test_blur_decimate_matches_fft(H, W, c, R):
    # Sec. II-A: D B(u) z is the circular convolution sampled at (ck, cl).
    z, u = rand(H, W), kern(R)
    ref = dense_ref.fft_conv(z, u)[::c, ::c]
    np.testing.assert_allclose(oracle.blur_decimate(z, u, c), ref,
                               rtol=0, atol=1e-12)


def test_blur_decimate_asymmetric_kernel_orientation():
    # A single off-centre tap u(i, j) = 1 at (i, j) = (1, -2) shifts the image:
    # (B z)(y, x) = z(y - 1, x + 2). Catches a flipped or transposed kernel.
    H, W, R = 12, 16, 3
    u = np.zeros((7, 7))
    u[1 + R, -2 + R] = 1.0
    z = rand(H, W)
    out = oracle.blur_decimate(z, u, 1)
    np.testing.assert_allclose(out, np.roll(np.roll(z, 1, axis=0), -2, axis=1),
                               atol=1e-14)


@pytest.mark.parametrize("H,W,c,R", [(24, 32, 4, 3), (20, 28, 4, 4),
                                     (16, 16, 4, 8)])
def test_blur_adjoint_identity(H, W, c, R):
    z, v, u = rand(H, W), rand(H // c, W // c), kern(R)
    lhs = np.vdot(oracle.blur_decimate(z, u, c), v)
    rhs = np.vdot(z, oracle.blur_decimate_adj(v, u, c))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_blur_adjoint_matches_dense():
    H, W, c, R = 12, 16, 4, 2
    u, v = kern(R), rand(H // c, W // c)
    A = dense_ref.decimation_matrix(H, W, c) @ dense_ref.conv_matrix(u, H, W)
    np.testing.assert_allclose(oracle.blur_decimate_adj(v, u, c).ravel(),
                               A.T @ v.ravel(), atol=1e-12)


def test_laplacian():
    z = rand(11, 14)
    S = np.array([[0, -1, 0], [-1, 4, -1], [0, -1, 0]], dtype=float)
    np.testing.assert_allclose(oracle.laplacian(z),
                               ndimage.convolve(z, S, mode="wrap"), atol=1e-12)
    # L annihilates constants (Sec. II-C) and is symmetric.
    np.testing.assert_allclose(oracle.laplacian(np.full((7, 9), 3.5)), 0.0,
                               atol=1e-13)
    v = rand(11, 14)
    assert abs(np.vdot(oracle.laplacian(z), v) - np.vdot(z, oracle.laplacian(v))) < 1e-11


@pytest.mark.parametrize("r", [1, 2])
def test_pan_stats_bruteforce(r):
    H, W, eps = 7, 9, 0.3
    Y = rand(H, W) * 10
    st = oracle.pan_stats(Y, r, eps)
    S = np.array([[0, -1, 0], [-1, 4, -1], [0, -1, 0]], dtype=float)
    I = ndimage.convolve(Y, S, mode="wrap")
    np.testing.assert_allclose(st.I, I, atol=1e-11)
    for y in range(H):
        for x in range(W):
            win = np.array([I[(y + dy) % H, (x + dx) % W]
                            for dy in range(-r, r + 1) for dx in range(-r, r + 1)])
            assert st.mu[y, x] == pytest.approx(np.mean(win), abs=1e-11)
            assert st.var[y, x] == pytest.approx(np.var(win), abs=1e-9)
            assert st.s[y, x] == pytest.approx(1.0 / (np.var(win) + eps), rel=1e-10)


def test_box_filter_matches_scipy():
    a = rand(20, 24)
    for half in (0, 1, 3):
        np.testing.assert_allclose(
            oracle.box_filter(a, half),
            ndimage.uniform_filter(a, size=2 * half + 1, mode="wrap"), atol=1e-12)


@pytest.mark.parametrize("H,W,r", [(8, 8, 1), (12, 12, 1), (8, 10, 2)])
def test_matting_matches_dense_matrix(H, W, r):
    # Matrix-free M (He-Sun-Tang form) against the matrix of Eq. matting_matrix
    # assembled entry by entry.
    I, eps = rand(H, W) * 5, 0.7
    st = oracle.fbmp.PanStats(I, *_stats_of_guide(I, r, eps), r, eps)
    M = dense_ref.matting_matrix(I, r, eps)
    alpha = rand(H, W)
    np.testing.assert_allclose(oracle.matting_apply(alpha, st).ravel(),
                               M @ alpha.ravel(), atol=1e-10)


def _stats_of_guide(I, r, eps):
    H, W = I.shape
    mu, var = np.empty_like(I), np.empty_like(I)
    for y in range(H):
        for x in range(W):
            win = [I[(y + dy) % H, (x + dx) % W]
                   for dy in range(-r, r + 1) for dx in range(-r, r + 1)]
            mu[y, x], var[y, x] = np.mean(win), np.var(win)
    return mu, var, 1.0 / (var + eps)


def test_matting_is_levin_minimum():
    # Eq. pansharp_penalty: min over (a, c) of sum_j sum_{k in w_j}
    # [(alpha_k - a_j I_k - c_j)^2 + eps a_j^2] equals alpha^T M alpha.
    # Each window's minimum is found by a library least-squares solve.
    H, W, r, eps = 9, 8, 1, 0.4
    Y = rand(H, W) * 4
    st = oracle.pan_stats(Y, r, eps)
    alpha = rand(H, W)
    total = 0.0
    for y in range(H):
        for x in range(W):
            idx = [((y + dy) % H, (x + dx) % W)
                   for dy in range(-r, r + 1) for dx in range(-r, r + 1)]
            Iw = np.array([st.I[p] for p in idx])
            aw = np.array([alpha[p] for p in idx])
            nw = len(idx)
            A = np.vstack([np.stack([Iw, np.ones(nw)], axis=1),
                           [[np.sqrt(nw * eps), 0.0]]])
            rhs = np.concatenate([aw, [0.0]])
            sol, *_ = np.linalg.lstsq(A, rhs, rcond=None)
            total += np.sum((A @ sol - rhs) ** 2)
    quad = np.vdot(alpha, oracle.matting_apply(alpha, st))
    assert quad == pytest.approx(total, rel=1e-10)


def test_matting_null_space_and_symmetry():
    H, W, r = 16, 12, 1
    Y = rand(H, W) * 20
    st = oracle.pan_stats(Y, r, 1e-14)
    # Constants are annihilated for any eps.
    assert np.max(np.abs(oracle.matting_apply(np.full((H, W), 2.0), st))) < 1e-11
    # alpha = a I + c is annihilated as eps -> 0 (Levin et al., Thm. 1).
    alpha = 0.7 * st.I - 1.3
    out = oracle.matting_apply(alpha, st)
    assert np.max(np.abs(out)) < 1e-8 * np.max(np.abs(alpha))
    st = oracle.pan_stats(Y, r, 0.5)
    a, b = rand(H, W), rand(H, W)
    assert abs(np.vdot(oracle.matting_apply(a, st), b)
               - np.vdot(a, oracle.matting_apply(b, st))) < 1e-10


def test_prior_quadratic_form_through_alpha():
    # The CG loop's lean LLP walks sum alpha . (M alpha), alpha = L p, for
    # p^T (L^T M L p): equal because the periodic 5-point L is symmetric. On
    # the oracle's operators, with the sum written pixel by pixel here.
    H, W, r = 14, 10, 1
    st = oracle.pan_stats(rand(H, W) * 20, r, 0.3)
    p = rand(H, W)
    alpha = oracle.laplacian(p)
    m_alpha = oracle.matting_apply(alpha, st)
    lhs = np.vdot(p, oracle.laplacian(m_alpha))
    rhs = 0.0
    for y in range(H):
        for x in range(W):
            rhs += alpha[y, x] * m_alpha[y, x]
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert rhs > 0.0                                         # M is positive semidefinite


def test_guided_filter_textbook():
    # He et al.'s guided filter with explicit per-window fits, written here.
    H, W, r, eps = 10, 9, 1, 0.25
    Y = rand(H, W) * 3
    st = oracle.pan_stats(Y, r, eps)
    q = rand(H, W)
    I = st.I
    a = np.empty((H, W))
    c = np.empty((H, W))
    for y in range(H):
        for x in range(W):
            idx = [((y + dy) % H, (x + dx) % W)
                   for dy in range(-r, r + 1) for dx in range(-r, r + 1)]
            Iw = np.array([I[p] for p in idx])
            qw = np.array([q[p] for p in idx])
            cov = np.mean(Iw * qw) - Iw.mean() * qw.mean()
            a[y, x] = cov / (Iw.var() + eps)
            c[y, x] = qw.mean() - a[y, x] * Iw.mean()
    out = np.empty((H, W))
    for y in range(H):
        for x in range(W):
            idx = [((y + dy) % H, (x + dx) % W)
                   for dy in range(-r, r + 1) for dx in range(-r, r + 1)]
            out[y, x] = np.mean([a[p] for p in idx]) * I[y, x] + np.mean([c[p] for p in idx])
    np.testing.assert_allclose(oracle.guided_filter(q, st), out, atol=1e-12)
    # A filtering input that is exactly affine in the guide passes through
    # unchanged as eps -> 0.
    st0 = oracle.pan_stats(Y, r, 1e-14)
    q = 2.5 * st0.I + 0.75
    np.testing.assert_allclose(oracle.guided_filter(q, st0), q, atol=1e-8)


def _dense_A(H, W, c, u, Y, r, eps, lam):
    B = dense_ref.conv_matrix(u, H, W)
    D = dense_ref.decimation_matrix(H, W, c)
    L = dense_ref.laplacian_matrix(H, W)
    I = (L @ Y.ravel()).reshape(H, W)
    M = dense_ref.matting_matrix(I, r, eps)
    return B.T @ D.T @ D @ B + lam * L.T @ M @ L, B, D, L


def test_z0_system_matches_dense_and_is_spd():
    H, W, c, R, r, eps, lam = 16, 16, 4, 2, 1, 1.0, 2e-2
    rng = np.random.default_rng(7)
    u = kern(R, rng)
    Y = rng.random((H, W)) * 255
    A, *_ = _dense_A(H, W, c, u, Y, r, eps, lam)
    st = oracle.pan_stats(Y, r, eps)
    z = rng.standard_normal((H, W))
    np.testing.assert_allclose(oracle.apply_z0_system(z, u, c, st, lam).ravel(),
                               A @ z.ravel(), rtol=0, atol=1e-9 * np.abs(A).max())
    np.testing.assert_allclose(A, A.T, atol=1e-9 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0


def test_z0_cg_matches_dense_solve():
    # Eq. Z_ini_matting solved by the oracle's CG vs a LAPACK solve of the
    # independently assembled 1024 x 1024 system (32 x 32 torus).
    H, W, c, R, r, eps, lam = 32, 32, 4, 3, 1, 1.0, 2e-4
    rng = np.random.default_rng(11)
    u = kern(R, rng)
    Y = rng.random((H, W)) * 255
    X = rng.random((H // c, W // c)) * 255
    A, B, D, L = _dense_A(H, W, c, u, Y, r, eps, lam)
    b = B.T @ D.T @ X.ravel()
    ref = np.linalg.solve(A, b).reshape(H, W)
    st = oracle.pan_stats(Y, r, eps)
    ob = oracle.blur_decimate_adj(X, u, c)
    np.testing.assert_allclose(ob.ravel(), b, atol=1e-9 * np.abs(b).max())
    z, it, rel = oracle.cg_solve(0, ob, u, c, lam, st, tol=1e-13)
    assert rel < 1e-12
    assert oracle.rel_l2(z, ref) < 1e-9


def _zstep_fourier(rhs, u, c, lam):
    """Eq. Z_solution solved in the Fourier domain: per alias group of c^2
    frequencies the matrix is (1/c^2) v v^H + diag(t), v_j = conj(B_j),
    t_j = lam S_j^2; Sherman-Morrison, with the DC group (t_0 = 0) solved by
    substitution."""
    H, W = rhs.shape
    h, w = H // c, W // c
    R = u.shape[0] // 2
    k = np.zeros((H, W))
    for i in range(-R, R + 1):
        for j in range(-R, R + 1):
            k[i % H, j % W] += u[i + R, j + R]
    Bh = np.fft.fft2(k)
    wy = 2 * np.pi * np.arange(H)[:, None] / H
    wx = 2 * np.pi * np.arange(W)[None, :] / W
    Sh = 4 - 2 * np.cos(wy) - 2 * np.cos(wx)
    T = lam * Sh ** 2
    rh = np.fft.fft2(rhs)
    out = np.zeros((H, W), complex)
    for ky in range(h):
        for kx in range(w):
            ys = [ky + p * h for p in range(c) for q in range(c)]
            xs = [kx + q * w for p in range(c) for q in range(c)]
            v = np.conj(Bh[ys, xs])
            t = T[ys, xs]
            rr = rh[ys, xs]
            if t.min() > 0:
                ti = rr / t
                tv = v / t
                x = ti - tv * (np.vdot(v, ti)) / (c * c + np.vdot(v, tv))
            else:
                j0 = int(np.argmin(t))
                s = c * c * rr[j0] / v[j0]
                x = np.zeros(c * c, complex)
                for j in range(c * c):
                    if j != j0:
                        x[j] = (rr[j] - v[j] * s / (c * c)) / t[j]
                x[j0] = (s - sum(np.conj(v[j]) * x[j] for j in range(c * c) if j != j0)) / np.conj(v[j0])
            out[ys, xs] = x
    return np.real(np.fft.ifft2(out))


def test_zstep_cg_matches_fourier_and_dense():
    H, W, c, R, lam = 32, 32, 4, 3, 2e-4
    rng = np.random.default_rng(5)
    u = kern(R, rng)
    rhs = rng.standard_normal((H, W)) * 100
    z, it, rel = oracle.cg_solve(1, rhs, u, c, lam, None, tol=1e-13)
    assert rel < 1e-12
    np.testing.assert_allclose(z, _zstep_fourier(rhs, u, c, lam),
                               atol=1e-9 * np.abs(z).max())
    B = dense_ref.conv_matrix(u, H, W)
    D = dense_ref.decimation_matrix(H, W, c)
    L = dense_ref.laplacian_matrix(H, W)
    A = B.T @ D.T @ D @ B + lam * L.T @ L
    ref = np.linalg.solve(A, rhs.ravel()).reshape(H, W)
    assert oracle.rel_l2(z, ref) < 1e-9


def test_kernel_normal_equations():
    # E = D C(Y): column a of E is Y shifted by the tap a, then decimated;
    # E u must equal D B(u) Y (Eq. u_solve).
    H, W, c, R = 24, 20, 4, 2
    rng = np.random.default_rng(3)
    Y = rng.random((H, W)) * 255
    n = 2 * R + 1
    cols = []
    for i in range(-R, R + 1):
        for j in range(-R, R + 1):
            cols.append(np.roll(np.roll(Y, i, axis=0), j, axis=1)[::c, ::c].ravel())
    E = np.stack(cols, axis=1)
    u = kern(R, rng)
    np.testing.assert_allclose(E @ u.ravel(),
                               dense_ref.fft_conv(Y, u)[::c, ::c].ravel(),
                               rtol=1e-12, atol=1e-9)
    f = rng.random(E.shape[0]) * 255
    EtE, Etf = oracle.kernel_normal_eq(Y, f.reshape(H // c, W // c), c, R)
    np.testing.assert_allclose(EtE, E.T @ E, rtol=1e-12)
    np.testing.assert_allclose(Etf, E.T @ f, rtol=1e-12)
    assert EtE.shape == (n * n, n * n)
