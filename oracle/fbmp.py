"""FP64 oracle of the F-BMP method: kernel estimate (Algorithm 1) and the
per-band HRMS solve (Algorithm 2), following the paper's steps in its order.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Image-domain loops live in ``oracle.c`` (plain C, FP64); the small n x n
kernel-grid algebra (ADMM, Appendix A) is numpy in FP64, with numpy's FFT,
sort and dense linear algebra used as library steps.

Readings of passages the paper leaves open are marked READING; each one is
listed in the repository's design notes.
"""
from __future__ import annotations

import ctypes
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from ._clib import lib


def f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------
# Parameters (Sec. IV-F, "Parameter Setting")
# ----------------------------------------------------------------------------
@dataclass
class KernelParams:
    lambda_omega: float = 10.0
    l: int = 2            # READING: box half-width on the LR grid; paper silent
    alpha1: float = 1.0
    alpha2: float = 0.006
    mu1: float = 100.0
    mu2: float = 100.0
    mu3: float = 100.0
    rho: float = 0.5
    t_max: int = 10000
    th: float = 1e-5


@dataclass
class HrmsParams:
    lam: float = 2e-4
    r: int = 1
    eps: float = 1.0      # READING: never given; on the [0, 255] scale
    tol: float = 1e-12    # relative residual of each linear solve
    max_iter: int = 100000
    exact_weight: bool = False   # READING: Z-step weight lam (paper) or lam|w|
    stop_rule: int = 0    # Z0 CG stop: 0 relative residual <= tol; 1 the
                          # paper's relative change of the iterate < tol


# ----------------------------------------------------------------------------
# Image-domain operators (C)
# ----------------------------------------------------------------------------
def blur_decimate(z, u, c: int) -> np.ndarray:
    """D B(u) z (Sec. II-A)."""
    z, u = f64(z), f64(u)
    H, W = z.shape
    R = u.shape[0] // 2
    out = np.empty((H // c, W // c))
    lib().or_blur_decimate(z, H, W, u, R, c, out)
    return out


def blur_decimate_adj(v, u, c: int) -> np.ndarray:
    """B(u)^T D^T v."""
    v, u = f64(v), f64(u)
    h, w = v.shape
    R = u.shape[0] // 2
    out = np.empty((h * c, w * c))
    lib().or_blur_decimate_adj(v, h * c, w * c, u, R, c, out)
    return out


def laplacian(z) -> np.ndarray:
    """L z, the 5-point Laplacian S of Eq. reg2, circular."""
    z = f64(z)
    out = np.empty_like(z)
    lib().or_laplacian(z, z.shape[0], z.shape[1], out)
    return out


@dataclass
class PanStats:
    I: np.ndarray
    mu: np.ndarray
    var: np.ndarray
    s: np.ndarray
    r: int
    eps: float


def pan_stats(Y, r: int, eps: float) -> PanStats:
    """I = L Y, window mean, population variance, s = 1/(var + eps)
    (Algorithm 2 step 3; Eq. ac_h_compute)."""
    Y = f64(Y)
    H, W = Y.shape
    I, mu, var, s = (np.empty_like(Y) for _ in range(4))
    lib().or_pan_stats(Y, H, W, r, eps, I, mu, var, s)
    return PanStats(I, mu, var, s, r, eps)


def matting_apply(alpha, st: PanStats) -> np.ndarray:
    """M alpha for the matting matrix of I (Eq. matting_matrix)."""
    alpha = f64(alpha)
    out = np.empty_like(alpha)
    lib().or_matting_apply(alpha, st.I, st.mu, st.s, alpha.shape[0],
                           alpha.shape[1], st.r, out)
    return out


def guided_filter(q, st: PanStats) -> np.ndarray:
    """Guided filter of q with guide I (Eq. ac_h_compute): the L-hat of
    Eq. Z_solution when q = L Z0."""
    q = f64(q)
    out = np.empty_like(q)
    lib().or_guided_filter(q, st.I, st.mu, st.s, q.shape[0], q.shape[1],
                           st.r, out)
    return out


def box_filter(a, half: int) -> np.ndarray:
    """Unit-gain (2 half + 1)^2 box, circular (u1, u2 of Eq. objective3)."""
    a = f64(a)
    out = np.empty_like(a)
    lib().or_box_filter(a, a.shape[0], a.shape[1], half, out)
    return out


_ZERO = np.zeros(1)


def apply_z0_system(z, u, c: int, st: PanStats, lam: float) -> np.ndarray:
    """(B^T D^T D B + lam L^T M L) z (Eq. Z_ini_matting)."""
    z, u = f64(z), f64(u)
    out = np.empty_like(z)
    lib().or_apply_system(z.shape[0], z.shape[1], c, u, u.shape[0] // 2,
                          st.I, st.mu, st.s, st.r, lam, 0, z, out)
    return out


def apply_zstep_system(z, u, c: int, lam: float) -> np.ndarray:
    """(B^T D^T D B + lam L^T L) z (Eq. Z_solution)."""
    z, u = f64(z), f64(u)
    out = np.empty_like(z)
    lib().or_apply_system(z.shape[0], z.shape[1], c, u, u.shape[0] // 2,
                          _ZERO, _ZERO, _ZERO, 0, lam, 1, z, out)
    return out


def cg_solve(op: int, b, u, c: int, lam: float, st: PanStats | None,
             x0=None, tol: float = 1e-12, max_iter: int = 100000):
    """CG on the Z0 system (op 0) or the Z-step system (op 1).
    Returns (x, iterations, true relative residual)."""
    b, u = f64(b), f64(u)
    H, W = b.shape
    x = np.zeros_like(b) if x0 is None else f64(x0).copy()
    rel = ctypes.c_double(0.0)
    if st is None:
        I = mu = s = _ZERO
        r = 0
    else:
        I, mu, s, r = st.I, st.mu, st.s, st.r
    it = lib().or_cg(H, W, c, u, u.shape[0] // 2, I, mu, s, r, lam, op, b, x,
                     tol, max_iter, ctypes.byref(rel))
    return x, it, rel.value


def keys_cubic(x, a: float = -0.5):
    """Keys' cubic convolution kernel W(x) (Keys 1981, a = -0.5)."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    return np.where(x <= 1.0, (a + 2) * x ** 3 - (a + 3) * x ** 2 + 1,
                    np.where(x < 2.0, a * x ** 3 - 5 * a * x ** 2 + 8 * a * x - 4 * a, 0.0))


def bicubic_up(X, c: int) -> np.ndarray:
    """Bicubic x c upsampling of the LR bands X (N x h x w, or h x w): the
    warm start of the Z0 solve. READING: HR pixel c k + phi lies on LR
    coordinate k + phi / c (phase 0, the samples D keeps), circular
    boundary; out(y, x) = sum_{i,j} W(t_y - i) W(t_x - j) X(k_y + i, k_x + j)
    over i, j in {-1, 0, 1, 2}, t = phi / c."""
    X = f64(X)
    if X.ndim == 2:
        return bicubic_up(X[None], c)[0]
    N, h, w = X.shape
    out = np.zeros((N, h * c, w * c))
    for py in range(c):
        wy = keys_cubic(py / c - np.arange(-1, 3))
        for px in range(c):
            wx = keys_cubic(px / c - np.arange(-1, 3))
            acc = np.zeros((N, h, w))
            for i in range(4):
                for j in range(4):
                    acc += wy[i] * wx[j] * np.roll(X, (-(i - 1), -(j - 1)), axis=(1, 2))
            out[:, py::c, px::c] = acc
    return out


def precond_apply(r, u, c: int, lam_gamma: float, tol: float = 1e-13) -> np.ndarray:
    """z = P^{-1} r with P = B^T D^T D B + lam_gamma L^T L, the operator of
    Eq. Z_solution at weight lam_gamma (L^T L from Eq. reg2 with M of
    Eq. Z_ini_matting replaced by gamma I). This is the preconditioner of
    the Z0 CG, an extension: the paper runs plain CG. Defined as the exact
    solve of P z = r, here the oracle's CG on that system to `tol`."""
    z, _, _ = cg_solve(1, r, u, c, lam_gamma, None, None, tol, 100000)
    return z


def pcg_solve(b, u, c: int, lam: float, st: PanStats, gamma: float, x0=None,
              tol: float = 1e-12, max_iter: int = 100000):
    """Preconditioned CG on the Z0 system of Eq. Z_ini_matting with the fixed
    SPD preconditioner P of precond_apply (P at weight lam * gamma): the
    textbook recurrence (Hestenes-Stiefel with z = P^{-1} r; e.g. Saad,
    Iterative Methods for Sparse Linear Systems, Alg. 9.1). It stops when the
    recursive residual ||r|| / ||b|| <= tol, the rule of the GPU solver.
    Returns (x, iterations, recursive relative residual)."""
    b, u = f64(b), f64(u)
    x = np.zeros_like(b) if x0 is None else f64(x0).copy()
    r = b - apply_z0_system(x, u, c, st, lam)
    bb = float(np.sum(b * b))
    if bb == 0.0:
        return x, 0, 0.0
    rel = float(np.sqrt(np.sum(r * r) / bb))
    if rel <= tol:
        return x, 0, rel
    z = precond_apply(r, u, c, lam * gamma)
    p = z.copy()
    rz = float(np.sum(r * z))
    for k in range(1, max_iter + 1):
        Ap = apply_z0_system(p, u, c, st, lam)
        alpha = rz / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        rel = float(np.sqrt(np.sum(r * r) / bb))
        if rel <= tol:
            return x, k, rel
        z = precond_apply(r, u, c, lam * gamma)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter, rel


def jacobi_diag(u, c: int, st: PanStats, lam: float) -> np.ndarray:
    """The diagonal of the Z0 operator A = B^T D^T D B + lam L^T M L of
    Eq. Z_ini_matting (L symmetric), pixel by pixel, from its definition.
    Data part: (B^T D^T D B)_{mm} is the sum over LR sites q of (D B)_{qm}^2;
    pixel m = (y, x) meets site (k, l) through the tap (c k - y, c l - x), so
    it is the sum of u(i, j)^2 over the taps with i = -y and j = -x mod c.
    Prior part: (L M L)_{mm} = sum over a, b in the 5-point stencil of m of
    L_{ma} M_{ab} L_{bm}, with M_{ab} the sum over the windows w_k holding
    both a and b of delta_ab - (1 + (I_a - mu_k)(I_b - mu_k) s_k) / |w|
    (Eq. matting_matrix, denominator sigma_k^2 + eps). The Jacobi
    preconditioner of the Z0 CG is its inverse (an extension: the paper runs
    plain CG)."""
    u = f64(u)
    H, W = st.I.shape
    R = u.shape[0] // 2
    y = np.arange(H)[:, None]
    x = np.arange(W)[None, :]
    data = np.zeros((H, W))
    for i in range(-R, R + 1):
        for j in range(-R, R + 1):
            hit = ((y + i) % c == 0) & ((x + j) % c == 0)
            data += np.where(hit, u[i + R, j + R] ** 2, 0.0)
    r = st.r
    nw = float((2 * r + 1) ** 2)

    def at(a, dy, dx):   # value at pixel (y + dy, x + dx) on the torus
        return np.roll(a, (-dy, -dx), axis=(0, 1))

    stencil = [((0, 0), 4.0), ((-1, 0), -1.0), ((1, 0), -1.0), ((0, -1), -1.0), ((0, 1), -1.0)]
    prior = np.zeros((H, W))
    for da, la in stencil:
        Ia = at(st.I, *da)
        for db, lb in stencil:
            Ib = at(st.I, *db)
            Mab = np.zeros((H, W))
            for ky in range(-r - 1, r + 2):
                for kx in range(-r - 1, r + 2):
                    inside = all(abs(k - d) <= r for k, d in ((ky, da[0]), (kx, da[1]),
                                                              (ky, db[0]), (kx, db[1])))
                    if not inside:
                        continue
                    mu_k, s_k = at(st.mu, ky, kx), at(st.s, ky, kx)
                    Mab += (1.0 if da == db else 0.0) - (1.0 + (Ia - mu_k) * (Ib - mu_k) * s_k) / nw
            prior += la * lb * Mab
    return data + lam * prior


def pcg_diag_solve(b, u, c: int, lam: float, st: PanStats, s, x0=None, tol: float = 1e-12,
                   max_iter: int = 100000):
    """Preconditioned CG on the Z0 system of Eq. Z_ini_matting with a diagonal
    preconditioner, P^{-1} = diag(s), s > 0 per pixel (an extension: the
    paper runs plain CG). The same textbook recurrence as pcg_solve with
    z = s * r. The stop rule is the recursive residual ||r|| / ||b|| <= tol.
    Returns (x, iterations, recursive relative residual)."""
    b, u, s = f64(b), f64(u), f64(s)
    if s.shape != b.shape or not np.all(s > 0.0):
        raise ValueError("s must be positive and shaped like b")
    x = np.zeros_like(b) if x0 is None else f64(x0).copy()
    r = b - apply_z0_system(x, u, c, st, lam)
    bb = float(np.sum(b * b))
    if bb == 0.0:
        return x, 0, 0.0
    rel = float(np.sqrt(np.sum(r * r) / bb))
    if rel <= tol:
        return x, 0, rel
    z = s * r
    p = z.copy()
    rz = float(np.sum(r * z))
    for k in range(1, max_iter + 1):
        Ap = apply_z0_system(p, u, c, st, lam)
        alpha = rz / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        rel = float(np.sqrt(np.sum(r * r) / bb))
        if rel <= tol:
            return x, k, rel
        z = s * r
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter, rel


def cg_relchange(b, u, c: int, lam: float, st: PanStats, x0=None, tol: float = 5e-5,
                 max_iter: int = 100000):
    """CG on the Z0 system of Eq. Z_ini_matting (textbook Hestenes-Stiefel)
    with the stop rule of Sec. IV-F: stop after the first iteration k whose
    relative change of the iterate in the Frobenius norm,
    ||x_k - x_(k-1)|| / ||x_k|| = |alpha| ||p|| / ||x_k||, is below tol.
    Before any iteration it stops only on an exact zero residual.
    Returns (x, iterations, recursive relative residual)."""
    b, u = f64(b), f64(u)
    x = np.zeros_like(b) if x0 is None else f64(x0).copy()
    r = b - apply_z0_system(x, u, c, st, lam)
    bb = float(np.sum(b * b))
    rr = float(np.sum(r * r))
    if bb == 0.0 or rr == 0.0:
        return x, 0, 0.0
    p = r.copy()
    for k in range(1, max_iter + 1):
        Ap = apply_z0_system(p, u, c, st, lam)
        alpha = rr / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.sum(r * r))
        change = abs(alpha) * float(np.linalg.norm(p)) / float(np.linalg.norm(x))
        if change < tol:
            return x, k, float(np.sqrt(rr_new / bb))
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, max_iter, float(np.sqrt(rr / bb))


# ----------------------------------------------------------------------------
# Alternative cross-channel priors (Sec. IV-D, Table III): the LLP's Laplacian
# replaced by other filters F_d; each keeps its own local affine model of
# F_d Z_i against the guide F_d Y, so the Z0 operator becomes
# B^T D^T D B + lam sum_d F_d^T M_d F_d and the Z step
# (B^T D^T D B + lam' sum_d F_d^T F_d) Z = B^T D^T X + lam' sum_d F_d^T L-hat_d.
# ----------------------------------------------------------------------------
PRIORS = ("llp", "lpf", "hpf", "lpp", "lgc")


def prior_filters(prior: str, u) -> list:
    """The filters F_d of a prior, on (2R+1)^2 grids with the convention of
    B(u) (tap (i, j) weighs z(y - i, x - j)). llp: the 5-point Laplacian;
    lpf: the blur kernel u (low-pass); hpf: delta - u (its complement); lpp:
    delta (the pixels); lgc: the horizontal and vertical differences
    z(y, x) - z(y, x - 1) and z(y, x) - z(y - 1, x) (Eq. reg2_lgc)."""
    u = f64(u)
    R = u.shape[0] // 2
    if prior == "llp":
        return [np.array([[0.0, -1.0, 0.0], [-1.0, 4.0, -1.0], [0.0, -1.0, 0.0]])]
    if prior == "lpf":
        return [u.copy()]
    if prior == "hpf":
        d = -u.copy()
        d[R, R] += 1.0
        return [d]
    if prior == "lpp":
        return [np.ones((1, 1))]
    if prior == "lgc":
        h = np.zeros((3, 3))
        h[1, 1], h[1, 2] = 1.0, -1.0
        v = np.zeros((3, 3))
        v[1, 1], v[2, 1] = 1.0, -1.0
        return [h, v]
    raise ValueError(prior)


def filt(z, F) -> np.ndarray:
    """F z, circular (B(F) of Sec. II-A without decimation)."""
    return blur_decimate(z, F, 1)


def filt_adj(z, F) -> np.ndarray:
    """F^T z."""
    return blur_decimate_adj(z, F, 1)


def guide_stats(I, r: int, eps: float) -> PanStats:
    """Window mean, population variance and s = 1/(var + eps) of a given
    guide image I over (2r+1)^2 circular windows."""
    I = f64(I)
    mu = box_filter(I, r)
    var = box_filter(I * I, r) - mu * mu
    return PanStats(I, mu, var, 1.0 / (var + eps), r, eps)


def prior_stats(Y, prior: str, u, r: int, eps: float) -> list:
    return [guide_stats(filt(Y, F), r, eps) for F in prior_filters(prior, u)]


def apply_z0_prior(z, u, c: int, filters, stats, lam: float) -> np.ndarray:
    """(B^T D^T D B + lam sum_d F_d^T M_d F_d) z."""
    out = blur_decimate_adj(blur_decimate(z, u, c), u, c)
    for F, st in zip(filters, stats):
        out += lam * filt_adj(matting_apply(filt(z, F), st), F)
    return out


def apply_zstep_prior(z, u, c: int, filters, lam: float) -> np.ndarray:
    """(B^T D^T D B + lam sum_d F_d^T F_d) z."""
    out = blur_decimate_adj(blur_decimate(z, u, c), u, c)
    for F in filters:
        out += lam * filt_adj(filt(z, F), F)
    return out


def cg_op(apply, b, x0=None, tol: float = 1e-12, max_iter: int = 100000):
    """Textbook CG (Hestenes-Stiefel) for an SPD operator given as a
    function; stops on the recursive relative residual. Returns (x, iters)."""
    b = f64(b)
    x = np.zeros_like(b) if x0 is None else f64(x0).copy()
    r = b - apply(x)
    bb = float(np.sum(b * b))
    rr = float(np.sum(r * r))
    if bb == 0.0 or np.sqrt(rr / bb) <= tol:
        return x, 0
    p = r.copy()
    for k in range(1, max_iter + 1):
        Ap = apply(p)
        alpha = rr / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.sum(r * r))
        if np.sqrt(rr_new / bb) <= tol:
            return x, k
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, max_iter


def solve_band_prior(x_lr, u, c: int, prior: str, stats, p: HrmsParams, z_init=None):
    """One band of Algorithm 2 under an alternative prior: Z0 by CG on
    apply_z0_prior, the per-filter guided filters L-hat_d of F_d Z0, then
    the Z step by CG."""
    filters = prior_filters(prior, u)
    b = blur_decimate_adj(x_lr, u, c)
    z0, it0 = cg_op(lambda z: apply_z0_prior(z, u, c, filters, stats, p.lam), b, z_init,
                    p.tol, p.max_iter)
    lam_z = p.lam * ((2 * p.r + 1) ** 2 if p.exact_weight else 1.0)
    rhs = b.copy()
    for F, st in zip(filters, stats):
        rhs += lam_z * filt_adj(guided_filter(filt(z0, F), st), F)
    z, it1 = cg_op(lambda v: apply_zstep_prior(v, u, c, filters, lam_z), rhs, z0, p.tol,
                   p.max_iter)
    return {"Z": z, "Z0": z0, "iters_z0": it0, "iters_z": it1}


def solve_hrms_prior(X, Y, u, c: int, prior: str, p: HrmsParams | None = None,
                     threads: int = 1):
    """Algorithm 2 over all bands under an alternative prior."""
    p = p or HrmsParams()
    X = f64(X)
    stats = prior_stats(Y, prior, u, p.r, p.eps)
    N = X.shape[0]

    def one(bd):
        return solve_band_prior(X[bd], u, c, prior, stats, p)

    if threads > 1:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            out = list(ex.map(one, range(N)))
    else:
        out = [one(bd) for bd in range(N)]
    return {"Z": np.stack([o["Z"] for o in out]), "Z0": np.stack([o["Z0"] for o in out]),
            "bands": out}


def kernel_normal_eq(Y, f, c: int, R: int):
    """E^T E and E^T f with E = D C(Y) (Eq. z_update, Eq. z_solution)."""
    Y, f = f64(Y), f64(f)
    H, W = Y.shape
    nn = (2 * R + 1) ** 2
    EtE = np.empty((nn, nn))
    Etf = np.empty(nn)
    lib().or_kernel_normal_eq(Y, H, W, c, R, f, EtE, Etf)
    return EtE, Etf


# ----------------------------------------------------------------------------
# Algorithm 2: the per-band HRMS solve
# ----------------------------------------------------------------------------
def solve_band(x_lr, u, c: int, st: PanStats, p: HrmsParams, z_init=None):
    """One band of Algorithm 2: Z0 (Eq. Z_ini_matting, by CG, stopped by
    p.stop_rule), then the A, C step (Eq. ac_h_compute) as a guided filter,
    then the Z step (Eq. Z_solution), solved exactly (CG to relative residual
    p.tol, or 1e-12 under the relative-change rule)."""
    b = blur_decimate_adj(x_lr, u, c)
    if p.stop_rule == 1:
        z0, it0, rel0 = cg_relchange(b, u, c, p.lam, st, z_init, p.tol, p.max_iter)
    else:
        z0, it0, rel0 = cg_solve(0, b, u, c, p.lam, st, z_init, p.tol, p.max_iter)
    lhat = guided_filter(laplacian(z0), st)
    lam_z = p.lam * ((2 * p.r + 1) ** 2 if p.exact_weight else 1.0)
    rhs = b + lam_z * laplacian(lhat)
    ztol = p.tol if p.stop_rule == 0 else 1e-12
    z, it1, rel1 = cg_solve(1, rhs, u, c, lam_z, None, z0, ztol, p.max_iter)
    return {"Z": z, "Z0": z0, "iters_z0": it0, "relres_z0": rel0,
            "iters_z": it1, "relres_z": rel1, "b": b, "lhat": lhat}


def solve_hrms(X, Y, u, c: int, p: HrmsParams | None = None,
               threads: int = 1, z_init=None):
    """Algorithm 2 over all bands ("for i = 1..N, do in parallel"), with the
    bands spread over ``threads`` host threads. Returns the per-band dicts and
    the stacked Z, Z0."""
    p = p or HrmsParams()
    X = f64(X)
    st = pan_stats(Y, p.r, p.eps)
    N = X.shape[0]

    def one(b):
        zi = None if z_init is None else z_init[b]
        return solve_band(X[b], u, c, st, p, zi)

    if threads > 1:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            out = list(ex.map(one, range(N)))
    else:
        out = [one(b) for b in range(N)]
    return {"Z": np.stack([o["Z"] for o in out]),
            "Z0": np.stack([o["Z0"] for o in out]),
            "bands": out, "stats": st}


# ----------------------------------------------------------------------------
# Algorithm 1: blur kernel estimation
# ----------------------------------------------------------------------------
def estimate_omega(X, Y, c: int, l: int, lam_omega: float, bands=None):
    """Spectral weights (Eq. objective3): least squares of
    B(u1) X' omega against D B(u2) Y plus (lam_omega/2)||G omega||^2, G the
    first differences of consecutive weights, by its normal equations.
    READING: u1 is the (2l+1)^2 unit box on the LR grid and u2 the
    (2cl+1)^2 unit box on the HR grid (the same physical half-width)."""
    X = f64(X)
    if bands is not None:
        X = X[list(bands)]
    Np = X.shape[0]
    A = np.stack([box_filter(X[k], l).ravel() for k in range(Np)], axis=1)
    bvec = box_filter(Y, c * l)[::c, ::c].ravel()
    G = np.zeros((max(Np - 1, 0), Np))
    for k in range(Np - 1):
        G[k, k], G[k, k + 1] = -1.0, 1.0
    lhs = A.T @ A + lam_omega * (G.T @ G)
    return np.linalg.solve(lhs, A.T @ bvec)


def simplex_project(v) -> np.ndarray:
    """Euclidean projection onto {s >= 0, sum s = 1} (Eq. simplex), by the
    sort-based method of Wang and Carreira-Perpinan (2013)."""
    v = f64(v).ravel()
    srt = np.sort(v)[::-1]
    css = np.cumsum(srt)
    j = np.arange(1, v.size + 1)
    rho = np.nonzero(srt + (1.0 - css) / j > 0)[0][-1] + 1
    tau = (1.0 - css[rho - 1]) / rho
    return np.maximum(v + tau, 0.0)


def shrink2(e, t: float) -> np.ndarray:
    """Row-wise group soft threshold, rows along axis 0 (Eq. x_update):
    max(||e|| - t, 0) e / ||e||."""
    nrm = np.sqrt(np.sum(e * e, axis=0))
    scale = np.where(nrm > t, (nrm - t) / np.where(nrm > 0, nrm, 1.0), 0.0)
    return e * scale


# Circular forward differences on the n x n kernel grid (READING: circular,
# as the FFT diagonalisation of Appendix A requires):
#   (Dh u)(i, j) = u(i, j+1) - u(i, j),  (Dv u)(i, j) = u(i+1, j) - u(i, j).
def Dh(a):
    return np.roll(a, -1, axis=1) - a


def Dv(a):
    return np.roll(a, -1, axis=0) - a


def DhT(a):
    return np.roll(a, 1, axis=1) - a


def DvT(a):
    return np.roll(a, 1, axis=0) - a


def grad(u):
    """nabla u = [Dh u, Dv u] (Eq. reg1)."""
    return np.stack([Dh(u), Dv(u)])


def sym_grad(p1, p2):
    """E(p) = [Dh p1, (Dv p1 + Dh p2)/2, (Dv p1 + Dh p2)/2, Dv p2] (Eq. reg1)."""
    m = 0.5 * (Dv(p1) + Dh(p2))
    return np.stack([Dh(p1), m, m, Dv(p2)])


def det3(a):
    """|.| of Appendix A, elementwise over frequencies."""
    return (a[0][0] * a[1][1] * a[2][2] + a[0][1] * a[1][2] * a[2][0]
            + a[0][2] * a[1][0] * a[2][1] - a[0][2] * a[1][1] * a[2][0]
            - a[0][1] * a[1][0] * a[2][2] - a[0][0] * a[2][1] * a[1][2])


def up_system_symbols(n: int, kp: KernelParams):
    """Fourier symbols of the {u, p} block system (Eq. block_toeplitz), with
    the mu3 coupling to z added to d1 (READING: the {u,p} argmin of
    Eq. subproblems omits the (mu3/2)||z - u - Lambda3||^2 term; without it
    d1 vanishes at DC and u is undetermined)."""
    k = np.arange(n)
    dh = (np.exp(2j * np.pi * k / n) - 1.0)[None, :] * np.ones((n, 1))
    dv = (np.exp(2j * np.pi * k / n) - 1.0)[:, None] * np.ones((1, n))
    a1, a2 = kp.alpha1 * kp.mu1, kp.alpha2 * kp.mu2
    d1 = a1 * (np.abs(dh) ** 2 + np.abs(dv) ** 2) + kp.mu3
    d2 = a1 + a2 * np.abs(dh) ** 2 + 0.5 * a2 * np.abs(dv) ** 2
    d3 = a1 + a2 * np.abs(dv) ** 2 + 0.5 * a2 * np.abs(dh) ** 2
    d4 = -a1 * dh
    d5 = -a1 * dv
    d6 = 0.5 * a2 * np.conj(dh) * dv
    return [[d1 + 0j, np.conj(d4), np.conj(d5)],
            [d4, d2 + 0j, np.conj(d6)],
            [d5, d6, d3 + 0j]]


def up_rhs(x, y, z, L1, L2, L3, kp: KernelParams):
    """B1, B2, B3 of Appendix A (with + mu3 (z - Lambda3) in B1). The two
    middle columns of y and Lambda2 enter through their mean, which equals
    either one when they agree."""
    a1, a2 = kp.alpha1 * kp.mu1, kp.alpha2 * kp.mu2
    q = y - L2
    q23 = 0.5 * (q[1] + q[2])
    B1 = a1 * (DhT(x[0] - L1[0]) + DvT(x[1] - L1[1])) + kp.mu3 * (z - L3)
    B2 = a1 * (L1[0] - x[0]) + a2 * (DhT(q[0]) + DvT(q23))
    B3 = a1 * (L1[1] - x[1]) + a2 * (DvT(q[3]) + DhT(q23))
    return B1, B2, B3


def up_solve(x, y, z, L1, L2, L3, kp: KernelParams):
    """{u, p} subproblem by FFT and Cramer's rule (Eq. u_p_solution)."""
    n = z.shape[0]
    S = up_system_symbols(n, kp)
    Bh = [np.fft.fft2(B) for B in up_rhs(x, y, z, L1, L2, L3, kp)]
    den = det3(S)
    out = []
    for col in range(3):
        M = [[Bh[row] if j == col else S[row][j] for j in range(3)]
             for row in range(3)]
        out.append(np.real(np.fft.ifft2(det3(M) / den)))
    return out  # u, p1, p2


@dataclass
class AdmmResult:
    kernel: np.ndarray          # z at exit, in the simplex
    u: np.ndarray
    iters: int
    converged: bool
    primal: dict = field(default_factory=dict)


def admm(EtE, Etf, R: int, kp: KernelParams | None = None) -> AdmmResult:
    """Algorithm 1's loop (Eq. subproblems, generalized ADMM).
    READING (init, paper silent): u0 = z0 = 1/n^2, p, x, y, Lambdas = 0.
    READING (order): the {u,p} step uses the x, y, z just computed.
    READING (output): the kernel returned is z, which lies in the simplex."""
    kp = kp or KernelParams()
    n = 2 * R + 1
    nn = n * n
    Q = np.linalg.inv(f64(EtE) + kp.mu3 * np.eye(nn))
    Etf = f64(Etf)
    u = np.full((n, n), 1.0 / nn)
    z = u.copy()
    p1 = np.zeros((n, n))
    p2 = np.zeros((n, n))
    x = np.zeros((2, n, n))
    y = np.zeros((4, n, n))
    L1 = np.zeros((2, n, n))
    L2 = np.zeros((4, n, n))
    L3 = np.zeros((n, n))
    it, conv = 0, False
    for t in range(kp.t_max):
        x = shrink2(grad(u) - np.stack([p1, p2]) + L1, 1.0 / kp.mu1)
        y = shrink2(sym_grad(p1, p2) + L2, 1.0 / kp.mu2)
        z = simplex_project(Q @ (Etf + kp.mu3 * (u + L3).ravel())).reshape(n, n)
        u_new, p1, p2 = up_solve(x, y, z, L1, L2, L3, kp)
        L1 = L1 + kp.rho * (grad(u_new) - np.stack([p1, p2]) - x)
        L2 = L2 + kp.rho * (sym_grad(p1, p2) - y)
        L3 = L3 + kp.rho * (u_new - z)
        change = np.linalg.norm(u - u_new) / np.linalg.norm(u_new)
        u = u_new
        it = t + 1
        if change < kp.th:
            conv = True
            break
    primal = {
        "x": float(np.linalg.norm(grad(u) - np.stack([p1, p2]) - x)),
        "y": float(np.linalg.norm(sym_grad(p1, p2) - y)),
        "z": float(np.linalg.norm(u - z)),
    }
    return AdmmResult(z, u, it, conv, primal)


def estimate_kernel(X, Y, c: int, R: int, kp: KernelParams | None = None,
                    omega=None, bands=None):
    """Algorithm 1: omega (Eq. objective3) unless given, then E^T E, E^T f
    and the ADMM loop. Returns (kernel n x n, omega, AdmmResult)."""
    kp = kp or KernelParams()
    X = f64(X)
    Xp = X if bands is None else X[list(bands)]
    if omega is None:
        omega = estimate_omega(Xp, Y, c, kp.l, kp.lambda_omega)
    f = np.tensordot(f64(omega), Xp, axes=1)
    EtE, Etf = kernel_normal_eq(Y, f, c, R)
    res = admm(EtE, Etf, R, kp)
    return res.kernel, f64(omega), res


def pansharpen(X, Y, c: int, R: int, kp: KernelParams | None = None,
               hp: HrmsParams | None = None, threads: int = 1, omega=None):
    """The two-stage scheme (Sec. III-C): Algorithm 1 once, then
    Algorithm 2 once, no outer loop."""
    kernel, omega, res = estimate_kernel(X, Y, c, R, kp, omega)
    out = solve_hrms(X, Y, kernel, c, hp, threads)
    out.update({"kernel": kernel, "omega": omega, "admm": res})
    return out


# ----------------------------------------------------------------------------
# Metrics used for reporting (Eq. psnr_def, Eq. relative_error_kernel)
# ----------------------------------------------------------------------------
def rel_l2(a, b) -> float:
    a, b = f64(a), f64(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def psnr(est, ref, border: int = 0) -> float:
    est, ref = f64(est), f64(ref)
    if border:
        est = est[..., border:-border, border:-border]
        ref = ref[..., border:-border, border:-border]
    mse = np.mean((est - ref) ** 2)
    return float(20.0 * np.log10(255.0 / np.sqrt(mse)))


def kernel_error_pct(est, ref) -> float:
    return 100.0 * rel_l2(est, ref)
