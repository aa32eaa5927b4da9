"""The form the benchmark times, element by element against the FP64 oracle.

The benchmark's solve: the FFT alias-group preconditioned CG (precond = 1)
started from the trained warm-start network (warm = 2), the all-FP32 Z step
(zstep_fp32 = 1), relative residual 1e-6, with the launch shapes and branch
count picked by the autotuner. It runs here
- through ps_pansharpen on a 512 x 512 crop of the 8-band 1024^2 workload
  scene (LRMS 8 x 128^2, 17 x 17 kernel, ratio 4), solved as its own
  periodic scene;
- through ps_pansharpen_batched on 256 x 256 crops of the first scenes of the
  64-scene uneven batch (seeds 3000 + k; their own band counts and kernel
  sizes).
Every band's Z (and, for the single scene, Z0) must lie within rel-L2 1e-3
of the oracle's (Algorithm 1, then Algorithm 2 with every linear system
solved by FP64 CG to 1e-11): the per-band tolerance the pipeline promises
for its mixed-precision, warm-started form. The measured values are printed.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2103_09943_gb300", "weights", "warm_cnn.npz")
TOL_BAND = 1e-3          # per HRMS band, against the FP64 oracle
C1_CROP = 512
C3_CROP = 256
C3_SCENES = 3


def _oracle_run(sc):
    cfg = sc["config"]
    return oracle.pansharpen(sc["lrms"], sc["pan"], cfg.ratio, cfg.R,
                             hp=oracle.HrmsParams(tol=1e-11), threads=cfg.bands)


@pytest.fixture(scope="module")
def crops():
    c1 = synth.crop_scene(synth.make_scene("c1"), C1_CROP)
    c3 = [synth.crop_scene(synth.make_scene(cfg), C3_CROP)
          for cfg in synth.make_batch_configs(64, 3000)[:C3_SCENES]]
    return c1, c3


@pytest.fixture(scope="module")
def oracle_refs(crops):
    # all scenes at once: every band of every scene on its own host thread
    c1, c3 = crops
    with ThreadPoolExecutor(max_workers=1 + len(c3)) as ex:
        futs = [ex.submit(_oracle_run, sc) for sc in [c1, *c3]]
        out = [f.result() for f in futs]
    return out[0], out[1:]


def _bench_form(api, net, **kw):
    return api.default_hrms_params(precond=1, warm=2, cnn_params=net.params.data_ptr(),
                                   zstep_fp32=1, tol=1e-6, **kw)


@pytest.fixture(scope="module")
def network(cuda):
    from paper_2103_09943_gb300.cnn import WarmStartNet
    assert os.path.exists(WEIGHTS), "trained warm-start weights are part of the package"
    return WarmStartNet.load(WEIGHTS, device=cuda)


def test_single_scene_bench_form_matches_oracle(cuda, crops, oracle_refs, network):
    from paper_2103_09943_gb300 import api
    c1, _ = crops
    ref, _ = oracle_refs
    cfg = c1["config"]
    hp = _bench_form(api, network)
    X, Y = to_dev(c1["lrms"], cuda), to_dev(c1["pan"], cuda)
    ws = api.workspace(cfg.bands, cfg.H, cfg.W, cfg.ratio, cfg.R, cuda, hp)
    K0, _, _ = api.estimate_kernel(X, Y, cfg.ratio, cfg.R, ws=ws, info=False)
    tuning = api.autotune(cfg.bands, cfg.H, cfg.W, cfg.ratio, cfg.R, hp.r, ws=ws, lrms=X,
                          pan=Y, kernel=K0)
    Z, K, kinfo, binfo = api.pansharpen(X, Y, cfg.ratio, cfg.R, hparams=hp, ws=ws)
    _, Z0, _ = api.solve_hrms(X, Y, K, cfg.ratio, hp, want_z0=True, ws=ws)
    Z, Z0, K = to_np(Z), to_np(Z0), to_np(K)
    assert kinfo.status == 0 and all(s == 0 for s in binfo.status), binfo
    ek = rel(K, ref["kernel"])
    ez = [rel(Z[b], ref["Z"][b]) for b in range(cfg.bands)]
    ez0 = [rel(Z0[b], ref["Z0"][b]) for b in range(cfg.bands)]
    print(f"\n{cfg.bands} x {C1_CROP}^2 crop, split {tuning['split']}, CG iters {binfo.iters}: "
          f"kernel {ek:.2e}; Z per band {['%.2e' % e for e in ez]}; "
          f"Z0 per band {['%.2e' % e for e in ez0]}")
    assert ek < 1e-4
    assert max(ez) < TOL_BAND
    assert max(ez0) < TOL_BAND


def test_batched_bench_form_matches_oracle(cuda, crops, oracle_refs, network):
    from paper_2103_09943_gb300 import api
    _, c3 = crops
    _, refs = oracle_refs
    hp = _bench_form(api, network)
    dev = [(to_dev(s["lrms"], cuda), to_dev(s["pan"], cuda), s["config"].R) for s in c3]
    b = api.Batch(dev, ratio=4, hparams=hp, estimate=True)
    for call in range(2):                 # the second launch reuses the graph
        kinfo, sinfo = b.run(info=True)
        for i, (sc, ref) in enumerate(zip(c3, refs)):
            cfg = sc["config"]
            assert kinfo[i].status == 0 and all(s == 0 for s in sinfo[i].status), (i, sinfo[i])
            Z = to_np(b.hrms[i])
            ek = rel(to_np(b.kernels[i]), ref["kernel"])
            ez = [rel(Z[k], ref["Z"][k]) for k in range(cfg.bands)]
            if call == 0:
                print(f"\nscene {i} ({cfg.bands} bands, {cfg.n}x{cfg.n}, {C3_CROP}^2 crop), "
                      f"CG iters {sinfo[i].iters}: kernel {ek:.2e}; Z per band "
                      f"{['%.2e' % e for e in ez]}")
            assert ek < 1e-4, i
            assert max(ez) < TOL_BAND, (i, ez)
