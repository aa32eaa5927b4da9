"""GPU parity of the bicubic warm start (Keys, a = -1/2, phase 0, circular)
against the FP64 oracle, and of the Z0 solve started from it: the stop rule is
unchanged, so the solution must match the cold start's."""
import numpy as np
import pytest

import oracle
import synth
from paper_2103_09943_gb300 import api, ops
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,h,w,c", [(3, 64, 64, 4), (2, 24, 36, 3), (1, 48, 32, 2),
                                     (2, 16, 12, 8)])
def test_bicubic_matches_oracle(cuda, N, h, w, c):
    rng = np.random.default_rng(N + h + w + c)
    X = rng.random((N, h, w)) * 255
    U = to_np(ops.bicubic_up(to_dev(X, cuda), c))
    ref = oracle.bicubic_up(X.astype(np.float32), c)
    assert U.shape == ref.shape
    assert np.abs(U - ref).max() < 2e-6 * np.abs(ref).max()


def test_warm_start_reaches_the_same_solution(cuda):
    sc = synth.make_scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    ref = oracle.solve_hrms(sc["lrms"], sc["pan"], sc["kernel"].astype(np.float64),
                            cfg.ratio, oracle.HrmsParams(tol=1e-11), threads=4)
    args = (to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda), to_dev(sc["kernel"], cuda),
            cfg.ratio)
    iters = {}
    for warm in (0, 1):
        hp = api.default_hrms_params(tol=1e-8, warm=warm)
        Z, Z0, info = api.solve_hrms(*args, hp, want_z0=True)
        assert all(s == 0 for s in info.status), info
        for b in range(cfg.bands):
            assert rel(to_np(Z0)[b], ref["Z0"][b]) < 1e-5, (warm, b)
            assert rel(to_np(Z)[b], ref["Z"][b]) < 1e-5, (warm, b)
        iters[warm] = info.iters
    # the bicubic start is closer to Z0 than zeros: never more iterations
    assert sum(iters[1]) <= sum(iters[0]) + cfg.bands, iters


def test_trained_network_saves_iterations(cuda):
    # a held-out scene of the 8-band 1024 x 1024 workload (seed outside the
    # training seeds 1000-2999): the committed network's start is closer to Z0
    # than the bicubic one and cuts the preconditioned CG's iterations, and
    # both starts reach the same Z0
    import os
    from dataclasses import replace
    from paper_2103_09943_gb300 import cnn
    wpath = os.path.join(os.path.dirname(cnn.__file__), "weights", "warm_cnn.npz")
    if not os.path.exists(wpath):
        pytest.skip("no trained weights")
    net = cnn.WarmStartNet.load(wpath, device=cuda)
    cfg = replace(synth.CONFIGS["c1"], seed=5005)
    sc = synth.make_scene(cfg)
    X, Y = to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda)
    K, _, _ = api.estimate_kernel(X, Y, cfg.ratio, cfg.R, info=False)
    out = {}
    for warm in (0, 2):
        hp = api.default_hrms_params(precond=1, warm=warm, cnn_params=net.params.data_ptr())
        _, Z0, info = api.solve_hrms(X, Y, K, cfg.ratio, hp, want_z0=True)
        assert all(s == 0 for s in info.status), info
        out[warm] = (to_np(Z0), float(np.mean(info.iters)))
    up = to_np(ops.bicubic_up(X, cfg.ratio))
    z_cnn = to_np(net.forward(ops.bicubic_up(X, cfg.ratio), Y, check=True))
    z0 = out[0][0]
    assert rel(z_cnn, z0) < 0.8 * rel(up, z0)
    assert out[2][1] < 0.85 * out[0][1], (out[0][1], out[2][1])
    assert rel(out[2][0], z0) < 1e-3


def test_heldout_warm_start_matches_oracle_on_crops(cuda):
    # The held-out scenes of the warm start's evaluation (seeds 5000 and up,
    # 8 x 2048^2 generated with the training generator's shape density):
    # 256 x 256 crops of the first two, each its own periodic scene, through
    # ps_pansharpen with the network's warm start and the preconditioned CG
    # (tolerance 1e-6), against the FP64 oracle (Algorithm 1, then Algorithm 2
    # with every linear system solved to 1e-11): every band within rel-L2
    # 1e-3, the bar of the mixed-precision, warm-started form.
    import os
    from concurrent.futures import ThreadPoolExecutor
    from paper_2103_09943_gb300 import cnn, eval_warm
    wpath = os.path.join(os.path.dirname(cnn.__file__), "weights", "warm_cnn.npz")
    net = cnn.WarmStartNet.load(wpath, device=cuda)
    crops = [synth.crop_scene(synth.make_scene(c), 256)
             for c in eval_warm.scene_configs(2, 2048, 5000)]

    def ref(sc):
        cfg = sc["config"]
        return oracle.pansharpen(sc["lrms"], sc["pan"], cfg.ratio, cfg.R,
                                 hp=oracle.HrmsParams(tol=1e-11), threads=cfg.bands)

    with ThreadPoolExecutor(max_workers=len(crops)) as ex:
        refs = list(ex.map(ref, crops))
    hp = api.default_hrms_params(precond=1, warm=2, cnn_params=net.params.data_ptr(),
                                 zstep_fp32=1, tol=1e-6)
    for sc, r in zip(crops, refs):
        cfg = sc["config"]
        Z, K, kinfo, info = api.pansharpen(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                           cfg.ratio, cfg.R, hparams=hp)
        assert all(s == 0 for s in info.status), info
        Z = to_np(Z)
        err = [rel(Z[b], r["Z"][b]) for b in range(cfg.bands)]
        print(f"\nheld-out seed {cfg.seed} 256^2 crop, CG iters {info.iters}: kernel "
              f"{rel(to_np(K), r['kernel']):.2e}; Z per band {['%.2e' % e for e in err]}")
        assert rel(to_np(K), r["kernel"]) < 1e-4
        assert max(err) < 1e-3
