"""Pins of the TGV^2 half of the oracle's ADMM (Algorithm 1) away from the
alpha -> 0 limit: the x and y shrinkage steps (Eq. x_update, Eq. y_update),
their thresholds 1/mu1 and 1/mu2, the Lambda1 and Lambda2 updates
(Eq. subproblems) and the way they enter the {u, p} step (Appendix A).

With E^T E = kappa I the printed z step (the unconstrained solve of
Eq. z_solution followed by the simplex projection) is the exact constrained
argmin, because the quadratic is isotropic. The ADMM's limit is then the
unique minimiser in u of Eq. u_solve,

    (kappa/2)||u||^2 - g^T u + alpha1 ||grad u - p||_{2,1}
                             + alpha2 ||E(p)||_{2,1} + I_S(u),   g = E^T f,

(strongly convex in u), which the test computes by an independent method:
the primal-dual algorithm of Chambolle and Pock (J. Math. Imaging Vis.
40, 2011, Alg. 1) on dense difference matrices written out from the
definitions of Eq. reg1. A planted mistake in any of those steps of the
oracle moves its result away from that minimiser (last test).
"""
import inspect

import numpy as np
import pytest

import oracle
import synth
from oracle import fbmp
from tests import dense_ref

PIN_ATOL = 1e-8            # max-abs difference of the kernels (entries ~1/n^2)
CP_ITERS = 20000


def _project_bisect(v, iters=64):
    # tau solves sum max(v + tau, 0) = 1 (monotone in tau): bisection.
    lo, hi = -v.max() - 1.0, -v.min() + 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if np.maximum(v + mid, 0).sum() > 1.0:
            hi = mid
        else:
            lo = mid
    return np.maximum(v + 0.5 * (lo + hi), 0)


def _operator(n):
    """K (u, p1, p2) = (grad u - p, E(p)): the 2 components of grad u - p and
    the 4 of the symmetrised derivative [Dh p1, (Dv p1 + Dh p2)/2,
    (Dv p1 + Dh p2)/2, Dv p2], each an n^2 block, pixel-major inside."""
    N = n * n
    Dh, Dv = dense_ref.grad_matrices(n)
    O, I = np.zeros((N, N)), np.eye(N)
    return np.block([[Dh, -I, O], [Dv, O, -I],
                     [O, Dh, O], [O, 0.5 * Dv, 0.5 * Dh], [O, 0.5 * Dv, 0.5 * Dh],
                     [O, O, Dv]])


def _chambolle_pock(n, kappa, g, a1, a2, iters=CP_ITERS):
    """min_w F(K w) + G(w), w = (u, p1, p2): F the two group norms (its
    conjugate's prox projects each pixel's 2- or 4-vector onto the ball of
    radius alpha), G = (kappa/2)||u||^2 - g^T u + I_S(u) (its prox scales,
    then projects onto the simplex; p is free). Steps tau = sigma = 0.99/||K||,
    extrapolation theta = 1."""
    N = n * n
    K = _operator(n)
    tau = sigma = 0.99 / np.linalg.norm(K, 2)
    w = np.zeros(3 * N)
    w[:N] = 1.0 / N
    wb = w.copy()
    q = np.zeros(6 * N)
    for _ in range(iters):
        q = q + sigma * (K @ wb)
        q1 = q[:2 * N].reshape(2, N)
        q1 /= np.maximum(1.0, np.sqrt((q1 ** 2).sum(0)) / a1)
        q2 = q[2 * N:].reshape(4, N)
        q2 /= np.maximum(1.0, np.sqrt((q2 ** 2).sum(0)) / a2)
        v = w - tau * (K.T @ q)
        wn = v.copy()
        wn[:N] = _project_bisect((v[:N] + tau * g) / (1.0 + tau * kappa))
        wb = 2.0 * wn - w
        w = wn
    return w[:N].reshape(n, n)


def _planted_problem(n, kappa, seed):
    # g = kappa u_target + noise, u_target a shifted Gaussian on the grid
    R = n // 2
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(n) - R, np.arange(n) - R, indexing="ij")
    ut = np.exp(-((i - 0.4) ** 2 + (j + 0.3) ** 2) / 2.0)
    ut /= ut.sum()
    return kappa * ut.ravel() + 0.5 * rng.standard_normal(n * n)


# (n, kappa, alpha1, alpha2, (mu1, mu2, mu3)): the paper's weights (Sec. IV-F)
# with its mu, the same with mu1 != mu2 (so a swapped threshold shows), and
# a larger alpha2 under which the first-order term stays active at the
# optimum (at the paper's weights p = grad u there, and x = 0)
CASES = {
    "paper": (5, 50.0, 1.0, 0.006, (100.0, 100.0, 100.0)),
    "paper_mu": (5, 50.0, 1.0, 0.006, (100.0, 40.0, 100.0)),
    "both_terms": (5, 50.0, 1.0, 0.5, (100.0, 40.0, 100.0)),
}


@pytest.fixture(scope="module")
def minimisers():
    out, solved = {}, {}
    for name, (n, kappa, a1, a2, _) in CASES.items():
        key = (n, kappa, a1, a2)          # mu does not change the minimiser
        if key not in solved:
            g = _planted_problem(n, kappa, seed=n)
            solved[key] = (g, _chambolle_pock(n, kappa, g, a1, a2))
        out[name] = solved[key]
    return out


def _admm(name, g, admm=None, t_max=50000):
    n, kappa, a1, a2, (m1, m2, m3) = CASES[name]
    kp = oracle.KernelParams(alpha1=a1, alpha2=a2, mu1=m1, mu2=m2, mu3=m3, t_max=t_max,
                             th=1e-13)
    return (admm or oracle.admm)(kappa * np.eye(n * n), g, n // 2, kp)


@pytest.mark.parametrize("name", list(CASES))
def test_admm_limit_is_the_tgv_minimiser(name, minimisers):
    g, u_star = minimisers[name]
    n, kappa = CASES[name][:2]
    res = _admm(name, g)
    assert res.converged
    assert np.abs(res.kernel - u_star).max() < PIN_ATOL
    # the regulariser matters here: the minimiser is far from the projection
    # of the data term's own minimiser
    assert np.abs(_project_bisect(g / kappa).reshape(n, n) - u_star).max() > 100 * PIN_ATOL


def test_primal_residuals_vanish_at_the_paper_weights():
    # Eq. subproblems' splitting constraints x = grad u - p, y = E(p), z = u
    # hold at convergence on real normal equations (the 4-band 256^2 scene,
    # the paper's alpha1, alpha2, mu), not only in the alpha -> 0 limit.
    sc = synth.make_scene("c0")
    cfg = sc["config"]
    kp = oracle.KernelParams(th=1e-11, t_max=50000)
    om = oracle.estimate_omega(sc["lrms"], sc["pan"], cfg.ratio, kp.l, kp.lambda_omega)
    f = np.tensordot(om, sc["lrms"].astype(np.float64), axes=1)
    EtE, Etf = oracle.kernel_normal_eq(sc["pan"], f, cfg.ratio, cfg.R)
    res = oracle.admm(EtE, Etf, cfg.R, kp)
    assert res.converged
    scale = np.linalg.norm(fbmp.grad(res.u))
    assert res.primal["x"] < 1e-6 * scale
    assert res.primal["y"] < 1e-6 * scale
    assert res.primal["z"] < 1e-6 * np.linalg.norm(res.u)


def _mutated_admm(edits):
    """oracle.fbmp.admm with the steps it calls re-defined from their source,
    each edit (function, text, replacement) applied first."""
    ns = dict(vars(fbmp))
    for fn in ("shrink2", "grad", "sym_grad", "up_system_symbols", "up_rhs", "up_solve",
               "admm"):
        src = inspect.getsource(getattr(fbmp, fn))
        for f2, old, new in edits:
            if f2 == fn:
                assert old in src, (fn, old)
                src = src.replace(old, new)
        exec(src, ns)
    return ns["admm"]


SLIPS = {
    "Lambda2 update sign": [("admm", "L2 = L2 + kp.rho", "L2 = L2 - kp.rho")],
    "Lambda1 update sign": [("admm", "L1 = L1 + kp.rho", "L1 = L1 - kp.rho")],
    "x shrink input": [("admm", "np.stack([p1, p2]) + L1, 1.0", "np.stack([p1, p2]) - L1, 1.0")],
    "x threshold": [("admm", "L1, 1.0 / kp.mu1", "L1, 1.0 / kp.mu2")],
    "y threshold": [("admm", "L2, 1.0 / kp.mu2", "L2, 1.0 / kp.mu1")],
    "E(p) middle term": [("sym_grad", "Dv(p1) + Dh(p2)", "Dv(p1) - Dh(p2)")],
    "B2 multiplier sign": [("up_rhs", "a1 * (L1[0] - x[0])", "a1 * (x[0] - L1[0])")],
    "B1 coupling to z": [("up_rhs", "kp.mu3 * (z - L3)", "kp.mu3 * (z + L3)")],
    "d2 middle weight": [("up_system_symbols", "a2 * np.abs(dh) ** 2 + 0.5 * a2",
                          "a2 * np.abs(dh) ** 2 + 1.0 * a2")],
}


@pytest.mark.parametrize("slip", list(SLIPS))
def test_a_planted_slip_fails_the_pin(slip, minimisers):
    admm = _mutated_admm(SLIPS[slip])
    caught = []
    for name in CASES:
        g, u_star = minimisers[name]
        try:
            with np.errstate(all="ignore"):
                res = _admm(name, g, admm, t_max=5000)   # unmutated: <= 400
            caught.append(not (res.converged and np.abs(res.kernel - u_star).max() < PIN_ATOL))
        except (ValueError, IndexError, FloatingPointError, np.linalg.LinAlgError):
            caught.append(True)          # the slip drove the iteration to NaN
    assert any(caught), slip
