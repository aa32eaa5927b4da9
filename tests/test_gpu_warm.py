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
