"""Pins of the oracle's preconditioner and preconditioned CG (an extension of
Eq. Z_ini_matting's solve: the paper runs plain CG).

P = B^T D^T D B + lam_gamma L^T L is checked against the independently
assembled dense matrix and against the per-alias-group Fourier closed form;
PCG against a LAPACK solve of the dense Z0 system."""
import numpy as np
import pytest

import oracle
import synth
from tests import dense_ref
from tests.test_oracle_operators import _dense_A, _zstep_fourier, kern


def _dense_P(H, W, c, u, lam_gamma):
    B = dense_ref.conv_matrix(u, H, W)
    D = dense_ref.decimation_matrix(H, W, c)
    L = dense_ref.laplacian_matrix(H, W)
    return B.T @ D.T @ D @ B + lam_gamma * L.T @ L


@pytest.mark.parametrize("H,W,c,R,lg", [(24, 24, 4, 2, 8e-4), (18, 12, 2, 3, 1e-2),
                                        (18, 27, 3, 1, 4.0)])
def test_precond_is_the_exact_inverse_of_dense_P(H, W, c, R, lg):
    rng = np.random.default_rng(H * W + c)
    u = kern(R, rng)
    P = _dense_P(H, W, c, u, lg)
    # SPD: symmetric, positive spectrum (the DC group is fixed by sum u = 1)
    np.testing.assert_allclose(P, P.T, atol=1e-12 * np.abs(P).max())
    assert np.linalg.eigvalsh(P).min() > 0
    r = rng.standard_normal((H, W)) * 50
    z = oracle.precond_apply(r, u, c, lg)
    ref = np.linalg.solve(P, r.ravel()).reshape(H, W)
    assert oracle.rel_l2(z, ref) < 1e-9


def test_precond_matches_fourier_group_solve():
    # the per-alias-group closed form (Sherman-Morrison, DC group by
    # substitution) is what the GPU kernels compute
    H, W, c, R, lg = 32, 48, 4, 3, 8e-4
    rng = np.random.default_rng(3)
    u = kern(R, rng)
    r = rng.standard_normal((H, W)) * 10
    np.testing.assert_allclose(oracle.precond_apply(r, u, c, lg), _zstep_fourier(r, u, c, lg),
                               atol=1e-9 * 10)


def test_precond_weight_matters():
    # a dropped or misplaced gamma changes the operator: P(lg1)^{-1} r differs
    # from P(lg2)^{-1} r by far more than the solve tolerance
    H, W, c, R = 24, 24, 4, 2
    rng = np.random.default_rng(5)
    u = kern(R, rng)
    r = rng.standard_normal((H, W))
    a = oracle.precond_apply(r, u, c, 2e-4)
    b = oracle.precond_apply(r, u, c, 8e-4)
    assert oracle.rel_l2(a, b) > 1e-2


def test_pcg_matches_dense_z0_solve():
    H, W, c, R, r, eps, lam = 32, 32, 4, 3, 1, 1.0, 2e-4
    rng = np.random.default_rng(11)
    u = kern(R, rng)
    Y = rng.random((H, W)) * 255
    X = rng.random((H // c, W // c)) * 255
    A, B, D, L = _dense_A(H, W, c, u, Y, r, eps, lam)
    b = B.T @ D.T @ X.ravel()
    ref = np.linalg.solve(A, b).reshape(H, W)
    st = oracle.pan_stats(Y, r, eps)
    z, it, rel = oracle.pcg_solve(b.reshape(H, W), u, c, lam, st, gamma=4.0, tol=1e-12)
    assert rel <= 1e-12
    assert oracle.rel_l2(z, ref) < 1e-9


def test_pcg_needs_fewer_iterations_on_a_scene():
    # same solution as plain CG to the same tolerance, in far fewer iterations
    # (64 x 64 crop of the 4-band 256^2 scene, 9 x 9 kernel, ratio 4)
    sc = synth.crop_scene(synth.make_scene(synth.CONFIGS["c0"]), 64)
    c, lam = 4, 2e-4
    u = sc["kernel"].astype(np.float64)
    st = oracle.pan_stats(sc["pan"], 1, 1.0)
    b = oracle.blur_decimate_adj(sc["lrms"][0], u, c)
    z_cg, it_cg, _ = oracle.cg_solve(0, b, u, c, lam, st, tol=1e-10)
    z_pcg, it_pcg, rel = oracle.pcg_solve(b, u, c, lam, st, gamma=4.0, tol=1e-10)
    assert rel <= 1e-10
    assert oracle.rel_l2(z_pcg, z_cg) < 1e-8
    assert it_pcg < it_cg / 2


def test_pcg_warm_start_at_solution_takes_no_iteration():
    sc = synth.crop_scene(synth.make_scene(synth.CONFIGS["c0"]), 32)
    c, lam = 4, 2e-4
    u = sc["kernel"].astype(np.float64)
    st = oracle.pan_stats(sc["pan"], 1, 1.0)
    b = oracle.blur_decimate_adj(sc["lrms"][1], u, c)
    z, _, _ = oracle.cg_solve(0, b, u, c, lam, st, tol=1e-13)
    _, it, rel = oracle.pcg_solve(b, u, c, lam, st, gamma=4.0, x0=z, tol=1e-9)
    assert it == 0 and rel <= 1e-9
