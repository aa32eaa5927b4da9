"""End-to-end parity of ps_pansharpen (Algorithm 1 then Algorithm 2) against
the FP64 oracle, and full-size checks on the 8-band 1024 x 1024 workload in
the launch configuration the benchmark times."""
import numpy as np
import pytest

import oracle
import synth
from paper_2103_09943_gb300 import api, ops
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def test_pansharpen_c0_end_to_end(cuda):
    sc = synth.make_scene("c0")
    cfg = sc["config"]
    ref = oracle.pansharpen(sc["lrms"], sc["pan"], cfg.ratio, cfg.R,
                            hp=oracle.HrmsParams(tol=1e-11), threads=4)
    hp = api.default_hrms_params(tol=1e-7)
    Z, k, kinfo, binfo = api.pansharpen(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                        cfg.ratio, cfg.R, hparams=hp)
    Z, k = to_np(Z), to_np(k)
    assert kinfo.status == 0
    assert rel(k, ref["kernel"]) < 1e-4
    for b in range(cfg.bands):
        assert rel(Z[b], ref["Z"][b]) < 1e-4
    # quality against the synthetic ground truth (context, not parity)
    assert oracle.psnr(Z, sc["hrms"], border=10) > 28.0


@pytest.fixture(scope="module")
def c1_run(cuda):
    sc = synth.make_scene("c1")
    cfg = sc["config"]
    hp = api.default_hrms_params()
    X, Y = to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda)
    Z, k, kinfo, binfo = api.pansharpen(X, Y, cfg.ratio, cfg.R, hparams=hp)
    # Z0 of the same kernel, for the residual checks
    _, Z0, info0 = api.solve_hrms(X, Y, k, cfg.ratio, hp, want_z0=True)
    return sc, hp, to_np(Z), to_np(Z0), to_np(k), kinfo, binfo


def test_c1_kernel_matches_oracle(c1_run):
    sc, hp, Z, Z0, k, kinfo, binfo = c1_run
    cfg = sc["config"]
    ref_k, ref_om, res = oracle.estimate_kernel(sc["lrms"], sc["pan"], cfg.ratio, cfg.R)
    assert rel(k, ref_k) < 1e-4
    assert kinfo.iters == pytest.approx(res.iters, abs=3)


def test_c1_z0_true_residual(c1_run):
    # Property at any size: the FP64 oracle's operator applied to the GPU's Z0
    # gives a true relative residual near the CG tolerance.
    sc, hp, Z, Z0, k, kinfo, binfo = c1_run
    cfg = sc["config"]
    st = oracle.pan_stats(sc["pan"], hp.r, hp.eps)
    for b in (0, cfg.bands - 1):
        rhs = oracle.blur_decimate_adj(sc["lrms"][b], k, cfg.ratio)
        res = rhs - oracle.apply_z0_system(Z0[b], k, cfg.ratio, st, hp.lambda_)
        assert np.linalg.norm(res) / np.linalg.norm(rhs) < 5 * hp.tol


def test_c1_zstep_exact_given_z0(c1_run):
    # The Z step solves its system exactly: the oracle's right-hand side built
    # from the GPU's Z0, minus the oracle's operator on the GPU's Z.
    sc, hp, Z, Z0, k, kinfo, binfo = c1_run
    cfg = sc["config"]
    st = oracle.pan_stats(sc["pan"], hp.r, hp.eps)
    for b in (1, cfg.bands - 2):
        lhat = oracle.guided_filter(oracle.laplacian(Z0[b]), st)
        rhs = oracle.blur_decimate_adj(sc["lrms"][b], k, cfg.ratio) + \
            hp.lambda_ * oracle.laplacian(lhat)
        res = rhs - oracle.apply_zstep_system(Z[b], k, cfg.ratio, hp.lambda_)
        assert np.linalg.norm(res) / np.linalg.norm(rhs) < 1e-5


def test_c1_sampled_stats(cuda, c1_run):
    sc = c1_run[0]
    I, mu, s = (to_np(t) for t in ops.pan_stats(to_dev(sc["pan"], cuda), 1, 1.0))
    rng = np.random.default_rng(0)
    H, W = sc["pan"].shape
    Y = sc["pan"].astype(np.float64)
    for _ in range(64):
        y, x = rng.integers(0, H), rng.integers(0, W)
        win = []
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                yy, xx = (y + dy) % H, (x + dx) % W
                win.append(4 * Y[yy, xx] - Y[(yy - 1) % H, xx] - Y[(yy + 1) % H, xx]
                           - Y[yy, (xx - 1) % W] - Y[yy, (xx + 1) % W])
        assert mu[y, x] == pytest.approx(np.mean(win), rel=1e-6, abs=1e-4)
        assert s[y, x] == pytest.approx(1.0 / (np.var(win) + 1.0), rel=1e-6)


def test_host_pipeline_matches_device_call(cuda):
    import torch
    sc = synth.make_scene("c0")
    cfg = sc["config"]
    pipe = api.HostPipeline(cfg.bands, cfg.H, cfg.W, cfg.ratio, cfg.R)
    hx = torch.from_numpy(sc["lrms"]).pin_memory()
    hy = torch.from_numpy(sc["pan"]).pin_memory()
    out = pipe(hx, hy)
    torch.cuda.synchronize()
    Z, _, _, _ = api.pansharpen(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda), cfg.ratio,
                                cfg.R)
    # FP64 atomics make the reduction order, hence the last bits, vary run to run
    assert rel(out.numpy(), to_np(Z)) < 1e-6


def test_paper_setting_29x29_motion_blur(cuda):
    # Sec. IV-F and Appendix B: a 29 x 29 kernel support, a Gaussian-times-
    # motion blur, plain CG from zeros with the relative-change stop rule.
    sc = synth.make_scene("p0")
    cfg = sc["config"]
    hp = api.default_hrms_params(tol=5e-5, stop_rule=1, precond=0, max_iter=5000)
    Z, k, kinfo, binfo = api.pansharpen(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                        cfg.ratio, cfg.R, hparams=hp)
    Z, k = to_np(Z), to_np(k)
    ref_k, _, res = oracle.estimate_kernel(sc["lrms"], sc["pan"], cfg.ratio, cfg.R)
    assert kinfo.status == 0
    assert k.shape == (29, 29)
    assert rel(k, ref_k) < 1e-4
    assert kinfo.iters == pytest.approx(res.iters, abs=3)
    ref = oracle.solve_hrms(sc["lrms"], sc["pan"], ref_k, cfg.ratio,
                            oracle.HrmsParams(tol=5e-5, stop_rule=1), threads=4)
    for b in range(cfg.bands):
        assert abs(binfo.iters[b] - ref["bands"][b]["iters_z0"]) <= 2, (b, binfo.iters)
        assert rel(Z[b], ref["Z"][b]) < 1e-4, b


def test_overlapped_call_equals_the_two_stages_in_sequence(cuda):
    # ps_pansharpen runs the kernel estimate on its own streams beside the
    # solve's PAN statistics and warm start; the result must be that of
    # ps_estimate_kernel followed by ps_solve_hrms on the caller's stream
    import os
    from paper_2103_09943_gb300.cnn import WarmStartNet
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    net = WarmStartNet.load(os.path.join(root, "paper_2103_09943_gb300", "weights",
                                         "warm_cnn.npz"), device=cuda)
    sc = synth.make_scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    X, Y = to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda)
    hp = api.default_hrms_params(tol=1e-7, warm=2, cnn_params=net.params.data_ptr())
    for _ in range(2):                      # the second call reuses the cached graphs
        Z, k, ki, si = api.pansharpen(X, Y, cfg.ratio, cfg.R, hparams=hp)
        k2, _, ki2 = api.estimate_kernel(X, Y, cfg.ratio, cfg.R)
        Z2, _, si2 = api.solve_hrms(X, Y, k2, cfg.ratio, hp)
        assert ki.iters == ki2.iters and ki.status == ki2.status == 0
        assert rel(to_np(k), to_np(k2)) < 1e-6
        for n in range(cfg.bands):
            assert abs(si.iters[n] - si2.iters[n]) <= 1, (si.iters, si2.iters)
        assert rel(to_np(Z), to_np(Z2)) < 1e-5
