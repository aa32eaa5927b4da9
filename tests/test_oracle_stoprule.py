"""Pins of the oracle's CG with the paper's stop rule (Sec. IV-F: stop when
the relative change of the iterate in the Frobenius norm is below the
threshold), against the oracle's C conjugate-gradient routine run for a fixed
number of iterations: an independent implementation of the same recurrence.
"""
import numpy as np
import pytest

import oracle

def _system(H=32, W=32, c=4, R=2, seed=77):
    rng = np.random.default_rng(seed)
    u = rng.random((2 * R + 1, 2 * R + 1))
    u /= u.sum()
    Y = rng.random((H, W)) * 255.0
    st = oracle.pan_stats(Y, 1, 1.0)
    x_lr = rng.random((H // c, W // c)) * 255.0
    b = oracle.blur_decimate_adj(x_lr, u, c)
    return b, u, c, st


def _iterate(b, u, c, st, lam, k):
    # k iterations of the C routine from zeros (tol 0: it never stops early)
    x, it, _ = oracle.cg_solve(0, b, u, c, lam, st, None, 0.0, k)
    assert it == k
    return x


@pytest.mark.parametrize("tol,seed", [(1e-2, 1), (1e-3, 2), (1e-3, 3)])
def test_relchange_stops_at_first_small_change(tol, seed):
    b, u, c, st = _system(seed=seed)
    lam = 2e-4
    x, k, _ = oracle.cg_relchange(b, u, c, lam, st, tol=tol)
    assert k >= 2
    xk, xk1, xk2 = (_iterate(b, u, c, st, lam, m) for m in (k, k - 1, k - 2))
    # the same iterate as the independent routine (the two sum in different
    # orders; CG on this ill-conditioned system amplifies that drift with the
    # iteration count, to ~1e-9 at 80 iterations)
    assert np.linalg.norm(x - xk) <= 1e-6 * np.linalg.norm(xk)
    # the rule holds at k and not one iteration earlier
    assert np.linalg.norm(xk - xk1) / np.linalg.norm(xk) < tol
    assert np.linalg.norm(xk1 - xk2) / np.linalg.norm(xk1) >= tol


def test_relchange_tighter_threshold_runs_longer_and_closer():
    b, u, c, st = _system(R=3)
    lam = 2e-4
    exact, _, rel = oracle.cg_solve(0, b, u, c, lam, st, None, 1e-13, 100000)
    errs, its = [], []
    for tol in (1e-2, 1e-4, 1e-6):
        x, k, _ = oracle.cg_relchange(b, u, c, lam, st, tol=tol)
        its.append(k)
        errs.append(np.linalg.norm(x - exact) / np.linalg.norm(exact))
    assert its[0] < its[1] < its[2]
    assert errs[0] > errs[1] > errs[2]


def test_relchange_zero_rhs_and_exact_start():
    b, u, c, st = _system()
    x, k, _ = oracle.cg_relchange(np.zeros_like(b), u, c, 2e-4, st)
    assert k == 0 and not x.any()
    exact, _, _ = oracle.cg_solve(0, b, u, c, 2e-4, st, None, 1e-14, 100000)
    # from the exact solution the first step is (near) zero: one iteration
    x, k, _ = oracle.cg_relchange(b, u, c, 2e-4, st, x0=exact, tol=1e-6)
    assert k <= 1
