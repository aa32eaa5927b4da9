"""GPU parity of the batched entry point (ps_pansharpen_batched): scenes of
uneven sizes, band counts and kernel supports in one graph launch give, scene
by scene, what the FP64 oracle gives (Algorithm 1 then Algorithm 2), and what
the one-scene calls give; kernels given or estimated; the network's warm
start inside the batch; per-scene finish times."""
import os
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2103_09943_gb300 import api
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2103_09943_gb300", "weights", "warm_cnn.npz")

# (bands, side, R): sides 2^a 3^b, LR grids 24..48 pixels, kernels 9x9 .. 13x13;
# the odd band count leaves half an image pair in the preconditioner's FFTs
SHAPES = [(4, 128, 4), (3, 192, 6), (8, 96, 4), (5, 144, 5)]


def _scenes():
    base = synth.CONFIGS["c0"]
    out = []
    for k, (N, side, R) in enumerate(SHAPES):
        cfg = replace(base, name=f"batch_{k}", bands=N, H=side, W=side, R=R, seed=4100 + k,
                      shapes=max(8, side * side // 2048))
        out.append(synth.make_scene(cfg))
    return out


@pytest.fixture(scope="module")
def scenes():
    return _scenes()


@pytest.fixture(scope="module")
def oracle_refs(scenes):
    """Algorithm 1 then Algorithm 2 on every scene by the FP64 oracle, every
    linear system solved to 1e-11."""
    out = []
    for sc in scenes:
        cfg = sc["config"]
        out.append(oracle.pansharpen(sc["lrms"], sc["pan"], cfg.ratio, cfg.R,
                                     hp=oracle.HrmsParams(tol=1e-11), threads=4))
    return out


@pytest.fixture(scope="module")
def batch_estimated(cuda, scenes):
    hp = api.default_hrms_params(tol=1e-7)
    dev = [(to_dev(s["lrms"], cuda), to_dev(s["pan"], cuda), s["config"].R) for s in scenes]
    b = api.Batch(dev, ratio=4, hparams=hp, estimate=True)
    kinfo, sinfo = b.run(info=True)
    return b, kinfo, sinfo, hp


def test_batch_matches_oracle(scenes, batch_estimated, oracle_refs):
    b, kinfo, sinfo, hp = batch_estimated
    for i, sc in enumerate(scenes):
        cfg = sc["config"]
        ref = oracle_refs[i]
        assert kinfo[i].status == 0, (i, kinfo[i].status)
        assert all(s == 0 for s in sinfo[i].status), (i, sinfo[i])
        assert rel(to_np(b.kernels[i]), ref["kernel"]) < 1e-4, i
        Z = to_np(b.hrms[i])
        for k in range(cfg.bands):
            assert rel(Z[k], ref["Z"][k]) < 1e-4, (i, k)


def test_batch_equals_single_scene_calls(cuda, scenes, batch_estimated):
    b, kinfo, sinfo, hp = batch_estimated
    for i, sc in enumerate(scenes):
        cfg = sc["config"]
        Z, k, ki, si = api.pansharpen(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                      cfg.ratio, cfg.R, hparams=hp)
        assert ki.iters == kinfo[i].iters
        assert rel(to_np(b.kernels[i]), to_np(k)) < 1e-6
        for n in range(cfg.bands):
            assert abs(si.iters[n] - sinfo[i].iters[n]) <= 1, (i, n)
        assert rel(to_np(b.hrms[i]), to_np(Z)) < 1e-5, i


def test_batch_rerun_reuses_graph_and_times_scenes(cuda, batch_estimated):
    b, kinfo, sinfo, hp = batch_estimated
    before = [t.clone() for t in b.hrms]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.run()
    e1.record()
    torch.cuda.synchronize()
    for x, y in zip(before, b.hrms):
        assert rel(to_np(y), to_np(x)) < 1e-6
    ms = b.scene_ms()
    assert len(ms) == b.count
    assert all(0.0 < t <= e0.elapsed_time(e1) * 1.05 + 0.5 for t in ms), ms


def test_batch_given_kernels_plain_fp32(cuda, scenes):
    # kernels given (the generator's), plain CG from zeros at a tight
    # tolerance: the plain FP32 bar against the oracle
    hp = api.default_hrms_params(tol=1e-8, precond=0, max_iter=5000)
    dev = [(to_dev(s["lrms"], cuda), to_dev(s["pan"], cuda), s["config"].R) for s in scenes]
    b = api.Batch(dev, ratio=4, hparams=hp, estimate=False)
    for i, s in enumerate(scenes):
        b.kernels[i].copy_(to_dev(s["kernel"], cuda))
    kinfo, sinfo = b.run(info=True)
    assert kinfo is None
    for i, sc in enumerate(scenes[:2]):
        cfg = sc["config"]
        ref = oracle.solve_hrms(sc["lrms"], sc["pan"], sc["kernel"].astype(np.float64),
                                cfg.ratio, oracle.HrmsParams(tol=1e-11), threads=4)
        Z = to_np(b.hrms[i])
        assert all(s == 0 for s in sinfo[i].status), sinfo[i]
        for k in range(cfg.bands):
            assert rel(Z[k], ref["Z"][k]) < 1e-5, (i, k)


def test_batch_network_warm_start(cuda, scenes, oracle_refs):
    from paper_2103_09943_gb300.cnn import WarmStartNet
    net = WarmStartNet.load(WEIGHTS, device=cuda)
    hp = api.default_hrms_params(tol=1e-7, warm=2, cnn_params=net.params.data_ptr())
    dev = [(to_dev(s["lrms"], cuda), to_dev(s["pan"], cuda), s["config"].R) for s in scenes]
    b = api.Batch(dev, ratio=4, hparams=hp, estimate=True)
    kinfo, sinfo = b.run(info=True)
    for i, sc in enumerate(scenes):
        cfg = sc["config"]
        # against the FP64 oracle: the warm start changes the start point,
        # not the solution
        Zb = to_np(b.hrms[i])
        assert rel(to_np(b.kernels[i]), oracle_refs[i]["kernel"]) < 1e-4, i
        for n in range(cfg.bands):
            assert rel(Zb[n], oracle_refs[i]["Z"][n]) < 1e-4, (i, n)
        # and against the one-scene call
        Z, k, ki, si = api.pansharpen(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                      cfg.ratio, cfg.R, hparams=hp)
        assert all(s == 0 for s in sinfo[i].status)
        for n in range(cfg.bands):
            assert abs(si.iters[n] - sinfo[i].iters[n]) <= 1, (i, n)
        assert rel(to_np(b.hrms[i]), to_np(Z)) < 1e-5, i


def test_batch_with_an_alternative_prior_and_the_paper_rule(cuda, scenes):
    # the batch runs whatever loop the parameters select: here the LGC prior
    # (plain CG) stopped by the paper's relative-change rule
    hp = api.default_hrms_params(precond=0, prior=4, stop_rule=1, tol=5e-5, max_iter=5000)
    dev = [(to_dev(s["lrms"], cuda), to_dev(s["pan"], cuda), s["config"].R) for s in scenes[:3]]
    b = api.Batch(dev, ratio=4, hparams=hp, estimate=True)
    kinfo, sinfo = b.run(info=True)
    for i, sc in enumerate(scenes[:3]):
        cfg = sc["config"]
        Z, k, ki, si = api.pansharpen(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                      cfg.ratio, cfg.R, hparams=hp)
        assert all(s == 0 for s in sinfo[i].status)
        for n in range(cfg.bands):
            assert abs(si.iters[n] - sinfo[i].iters[n]) <= 1, (i, n)
        assert rel(to_np(b.hrms[i]), to_np(Z)) < 1e-5, i


def test_batch_host_staging(cuda, scenes, batch_estimated):
    # The scenes' inputs copied from page-locked host tensors and every HRMS
    # copied back to page-locked host tensors by the batch graph itself: the
    # device inputs start as zeros, so a result equal to the device-only
    # batch's shows the copies ran before the work; the host HRMS is the
    # device HRMS of the same run, byte for byte.
    ref, _, _, hp = batch_estimated
    dev = [(torch.zeros(s["lrms"].shape, dtype=torch.float32, device=cuda),
            torch.zeros(s["pan"].shape, dtype=torch.float32, device=cuda), s["config"].R)
           for s in scenes]
    b = api.Batch(dev, ratio=4, hparams=hp, estimate=True)
    hin = [(torch.from_numpy(np.ascontiguousarray(s["lrms"], dtype=np.float32)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(s["pan"], dtype=np.float32)).pin_memory())
           for s in scenes]
    hout = b.stage_host(hin)
    kinfo, sinfo = b.run(info=True)
    for i in range(len(scenes)):
        assert kinfo[i].status == 0 and all(s == 0 for s in sinfo[i].status), i
        assert np.array_equal(hout[i].numpy(), to_np(b.hrms[i])), i
        assert rel(hout[i].numpy(), to_np(ref.hrms[i])) < 1e-6, i
    # a host pointer that is not page-locked is refused before any work
    pageable = np.zeros(scenes[0]["lrms"].shape, dtype=np.float32)
    b.scenes[0].h_lrms = pageable.ctypes.data
    with pytest.raises(api.PsError, match="status 1"):
        b.run()
