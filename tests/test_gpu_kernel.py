"""GPU parity of Algorithm 1 (blur kernel estimation) against the FP64
oracle: omega, E^T E / E^T f, the ADMM loop, and the whole estimate."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synth
from paper_2103_09943_gb300 import api, ops
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["c0"])
def test_omega(cuda, name):
    sc = synth.make_scene(name)
    cfg = sc["config"]
    kp = oracle.KernelParams()
    ref = oracle.estimate_omega(sc["lrms"], sc["pan"], cfg.ratio, kp.l, kp.lambda_omega)
    om = to_np(ops.omega(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda), cfg.ratio, kp.l,
                         kp.lambda_omega))
    assert rel(om, ref) < 1e-5


@pytest.mark.parametrize("H,c,R", [(256, 4, 4), (96, 4, 8), (120, 3, 2), (64, 2, 5)])
def test_kernel_normal_equations(cuda, H, c, R):
    rng = np.random.default_rng(H + R)
    N = 3
    Y = (rng.random((H, H)) * 255).astype(np.float32)
    X = (rng.random((N, H // c, H // c)) * 255).astype(np.float32)
    om = np.array([0.2, 0.5, 0.3], dtype=np.float32)
    ete, etf = ops.kernel_normal_eq(to_dev(X, cuda), to_dev(Y, cuda), to_dev(om, cuda), c, R)
    f = np.tensordot(om.astype(np.float64), X.astype(np.float64), axes=1)
    rE, rF = oracle.kernel_normal_eq(Y.astype(np.float64), f.astype(np.float32), c, R)
    # double-float accumulation of exact FP32 products: FP64-level agreement
    assert rel(to_np(ete), rE) < 1e-12
    # f is formed in FP32 on the device
    assert rel(to_np(etf), rF) < 1e-6


def test_admm_given_normal_equations(cuda):
    sc = synth.make_scene("c0")
    cfg = sc["config"]
    kp = oracle.KernelParams()
    om = oracle.estimate_omega(sc["lrms"], sc["pan"], cfg.ratio, kp.l, kp.lambda_omega)
    f = np.tensordot(om, sc["lrms"].astype(np.float64), axes=1)
    EtE, Etf = oracle.kernel_normal_eq(sc["pan"], f, cfg.ratio, cfg.R)
    res = oracle.admm(EtE, Etf, cfg.R, kp)
    import torch
    k, info = ops.admm(torch.from_numpy(EtE).to(cuda), torch.from_numpy(Etf).to(cuda), cfg.R)
    assert info.status == 0
    assert abs(info.iters - res.iters) <= 3
    assert rel(to_np(k), res.kernel) < 1e-4
    kn = to_np(k)
    assert kn.min() >= 0 and abs(kn.sum() - 1) < 1e-5


@pytest.mark.parametrize("name,R", [("c0", 4), ("c0", 6)])
def test_estimate_kernel(cuda, name, R):
    sc = synth.make_scene(replace(synth.CONFIGS[name], R=R))
    cfg = sc["config"]
    ref_k, ref_om, res = oracle.estimate_kernel(sc["lrms"], sc["pan"], cfg.ratio, R)
    k, om, info = api.estimate_kernel(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                      cfg.ratio, R)
    assert rel(to_np(om), ref_om) < 1e-5
    assert rel(to_np(k), ref_k) < 1e-4
    # and the estimate is close to the planted kernel (noisy data)
    assert oracle.kernel_error_pct(to_np(k), sc["kernel"]) < 15.0


def test_planted_kernel_recovery_on_gpu(cuda):
    # Noiseless data, omega given, weak regulariser: the GPU estimate recovers
    # the planted kernel (as the oracle does, see test_oracle_kernel).
    from tests.test_oracle_kernel import _noiseless_scene
    Z, Y, X, u_true, w = _noiseless_scene(H=128, R=3)
    kp = api.default_kernel_params(alpha1=1e-6, alpha2=1e-6, t_max=20000, th=1e-9)
    k, _, info = api.estimate_kernel(to_dev(X, cuda), to_dev(Y, cuda), 4, 3, kp,
                                     omega=to_dev(w, cuda))
    assert oracle.kernel_error_pct(to_np(k), u_true) < 1.0


def test_estimate_kernel_on_a_band_subset(cuda):
    # X' of Eq. objective1 a strict subset (bands 0 and 2 of the 4-band
    # scene): omega over X' (zeros for the other bands), f = X' omega, the
    # ADMM on the resulting normal equations; against the oracle's estimate
    # over the same subset. The same mask through ps_pansharpen, with omega
    # given (entries outside X' ignored), and per scene in a batch.
    sc = synth.make_scene("c0")
    cfg = sc["config"]
    bands = [0, 2]
    kp = api.default_kernel_params(band_mask=api.band_mask(bands))
    X, Y = to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda)
    ref_k, ref_om, res = oracle.estimate_kernel(sc["lrms"], sc["pan"], cfg.ratio, cfg.R,
                                                bands=bands)
    k, om, info = api.estimate_kernel(X, Y, cfg.ratio, cfg.R, kp)
    om, k = to_np(om), to_np(k)
    assert rel(om[bands], ref_om) < 1e-5
    assert np.all(om[[1, 3]] == 0.0)
    assert rel(k, ref_k) < 1e-4
    assert info.iters == pytest.approx(res.iters, abs=3)
    # the subset changes the estimate: omega over all bands differs
    _, om_all, _ = api.estimate_kernel(X, Y, cfg.ratio, cfg.R)
    assert rel(to_np(om_all)[bands], ref_om) > 1e-3
    # omega given: the entries of bands outside X' do not count
    om_in = to_dev(np.array([0.3, 5.0, 0.7, -2.0]), cuda)
    k2, om2, _ = api.estimate_kernel(X, Y, cfg.ratio, cfg.R, kp, omega=om_in)
    ref_k2, _, _ = oracle.estimate_kernel(sc["lrms"], sc["pan"], cfg.ratio, cfg.R,
                                          omega=np.array([0.3, 0.7]), bands=bands)
    assert rel(to_np(k2), ref_k2) < 1e-4
    assert np.allclose(to_np(om2), [0.3, 0.0, 0.7, 0.0])
    # ps_pansharpen and a batch (the scene's own mask) take the same X'
    _, k3, _, _ = api.pansharpen(X, Y, cfg.ratio, cfg.R, kparams=kp)
    assert rel(to_np(k3), k) < 1e-6
    b = api.Batch([(X, Y, cfg.R, api.band_mask(bands)), (X, Y, cfg.R)], cfg.ratio,
                  kparams=api.default_kernel_params())
    b.run()
    assert rel(to_np(b.kernels[0]), k) < 1e-6
    k_all, _, _ = api.estimate_kernel(X, Y, cfg.ratio, cfg.R)
    assert rel(to_np(b.kernels[1]), to_np(k_all)) < 1e-6
