"""GPU parity of the diagonal preconditioner of the Z0 CG (precond = 2, an
extension: the paper runs plain CG) against the FP64 oracle: with a given
diagonal, iterate for iterate against oracle.pcg_diag_solve; with a constant
one, against the plain CG; with the learned diagonal network, the same Z0
and HRMS as the oracle's solve; batched scenes as their single calls; a
non-finite diagonal stops its own band only. The network's weighted loss
and gradients match the oracle's."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import cnn as ocnn
from paper_2103_09943_gb300 import api, ops
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2103_09943_gb300", "weights")


def _smooth_positive(N, H, W, seed):
    """A seeded positive field spread over about e^2 (sums of plane waves)."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W] / np.array([H, W])[:, None, None]
    out = np.empty((N, H, W))
    for b in range(N):
        g = np.zeros((H, W))
        for _ in range(4):
            ky, kx = rng.integers(1, 6, 2)
            g += np.sin(2 * np.pi * (ky * y + kx * x) + rng.uniform(0, 2 * np.pi))
        out[b] = np.exp(0.25 * g)
    return out


@pytest.fixture(scope="module")
def c0():
    sc = synth.make_scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    ref = oracle.solve_hrms(sc["lrms"], sc["pan"], sc["kernel"].astype(np.float64),
                            cfg.ratio, oracle.HrmsParams(tol=1e-11), threads=4)
    return sc, ref


def _diag_net(cuda):
    from paper_2103_09943_gb300.cnn import WarmStartNet
    path = os.path.join(WEIGHTS, "diag_cnn.npz")
    if os.path.exists(path):
        return WarmStartNet.load(path, device=cuda)
    net = WarmStartNet(seed=17, device=cuda)
    net.params[-1] = 1.0
    return net


def test_given_diagonal_follows_the_oracle(cuda, c0):
    sc, _ = c0
    cfg = sc["config"]
    N, H, W, c = cfg.bands, cfg.H, cfg.W, cfg.ratio
    s = _smooth_positive(N, H, W, 91)
    sd = to_dev(s, cuda)
    u = sc["kernel"].astype(np.float64)
    st = oracle.pan_stats(sc["pan"], 1, 1.0)
    tol = 1e-5
    hp = api.default_hrms_params(tol=tol, precond=2, precond_diag=sd.data_ptr())
    _, Z0, info = api.solve_hrms(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                 to_dev(sc["kernel"], cuda), c, hp, want_z0=True)
    Z0 = to_np(Z0)
    for b in range(N):
        rhs = oracle.blur_decimate_adj(sc["lrms"][b], u, c)
        z, it, r = oracle.pcg_diag_solve(rhs, u, c, 2e-4, st, s[b], tol=tol)
        assert info.status[b] == 0, info
        assert abs(info.iters[b] - it) <= max(2, it // 30), (b, info.iters[b], it)
        assert rel(Z0[b], z) < 2e-4, b


def test_constant_diagonal_is_the_plain_cg(cuda, c0):
    sc, ref = c0
    cfg = sc["config"]
    args = (to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda), to_dev(sc["kernel"], cuda),
            cfg.ratio)
    sd = torch.full((cfg.bands, cfg.H, cfg.W), 3.0, device=cuda)
    _, Zp, ip = api.solve_hrms(*args, api.default_hrms_params(tol=1e-7, precond=0),
                               want_z0=True)
    _, Zd, idg = api.solve_hrms(*args, api.default_hrms_params(tol=1e-7, precond=2,
                                                              precond_diag=sd.data_ptr()),
                                want_z0=True)
    for b in range(cfg.bands):
        assert abs(ip.iters[b] - idg.iters[b]) <= 1, (ip, idg)
    assert rel(to_np(Zd), to_np(Zp)) < 1e-5


@pytest.mark.parametrize("warm", [0, 2])
def test_learned_diagonal_reaches_the_oracle(cuda, c0, warm):
    from paper_2103_09943_gb300.cnn import WarmStartNet
    sc, ref = c0
    cfg = sc["config"]
    dnet = _diag_net(cuda)
    kw = dict(tol=1e-8, max_iter=5000, precond=2, diag_params=dnet.params.data_ptr(), warm=warm)
    if warm == 2:
        wnet = WarmStartNet.load(os.path.join(WEIGHTS, "warm_cnn.npz"), device=cuda)
        kw["cnn_params"] = wnet.params.data_ptr()
    hp = api.default_hrms_params(**kw)
    Z, Z0, info = api.solve_hrms(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                 to_dev(sc["kernel"], cuda), cfg.ratio, hp, want_z0=True)
    assert all(s == 0 for s in info.status), info
    assert all(x <= 1e-8 * 1.0001 for x in info.rel_residual), info
    Z, Z0 = to_np(Z), to_np(Z0)
    for b in range(cfg.bands):
        assert rel(Z0[b], ref["Z0"][b]) < 1e-5, b
        assert rel(Z[b], ref["Z"][b]) < 1e-5, b


def test_learned_diagonal_batched_equals_single_calls(cuda):
    from dataclasses import replace
    dnet = _diag_net(cuda)
    hp = api.default_hrms_params(tol=1e-7, precond=2, diag_params=dnet.params.data_ptr())
    scenes = [synth.make_scene(replace(synth.CONFIGS["c0"], name=f"d{k}", bands=N, H=side,
                                       W=side, R=R, seed=4300 + k, shapes=12))
              for k, (N, side, R) in enumerate([(4, 128, 4), (3, 192, 6)])]
    dev = [(to_dev(s["lrms"], cuda), to_dev(s["pan"], cuda), s["config"].R) for s in scenes]
    b = api.Batch(dev, ratio=4, hparams=hp, estimate=True)
    _, sinfo = b.run(info=True)
    for i, sc in enumerate(scenes):
        cfg = sc["config"]
        Z, _, _, si = api.pansharpen(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                     cfg.ratio, cfg.R, hparams=hp)
        assert all(s == 0 for s in sinfo[i].status)
        for n in range(cfg.bands):
            assert abs(si.iters[n] - sinfo[i].iters[n]) <= 1, (i, n)
        assert rel(to_np(b.hrms[i]), to_np(Z)) < 1e-5, i


def test_nonfinite_diagonal_stops_its_band_only(cuda, c0):
    sc, ref = c0
    cfg = sc["config"]
    s = _smooth_positive(cfg.bands, cfg.H, cfg.W, 5)
    s[1, 10, 20] = np.nan
    sd = to_dev(s, cuda)
    hp = api.default_hrms_params(tol=1e-8, precond=2, precond_diag=sd.data_ptr())
    _, Z0, info = api.solve_hrms(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                 to_dev(sc["kernel"], cuda), cfg.ratio, hp, want_z0=True)
    assert info.status[1] == 6, info                               # non-finite
    Z0 = to_np(Z0)
    for b in (0, 2, 3):
        assert info.status[b] == 0, info
        assert rel(Z0[b], ref["Z0"][b]) < 1e-5, b


def test_weighted_loss_and_gradients_match_oracle(cuda):
    from paper_2103_09943_gb300.cnn import WarmStartNet, init_params, split_params
    rng = np.random.default_rng(31)
    B, H, W = 2, 24, 40
    p = init_params(9)
    parts = split_params(p)
    parts[-1][0][...] *= 10.0
    for _, bb in parts:
        bb[...] = rng.standard_normal(bb.shape) * 0.05
    up = (rng.random((B, H, W)) * 255).astype(np.float32)
    pan = (rng.random((B, H, W)) * 255).astype(np.float32)
    target = (up + rng.standard_normal((B, H, W)) * 20).astype(np.float32)
    weight = (rng.random((B, H, W)) * 2.0).astype(np.float32)
    weight[0, :4] = 0.0
    net = WarmStartNet(params=p, device=cuda)
    dev = lambda a: torch.from_numpy(a).to(cuda)
    loss = net.loss_grad(dev(up), dev(pan), dev(target), weight=dev(weight))
    grad = net.grad.double().cpu().numpy()
    ps = [(w.astype(np.float64), b.astype(np.float64)) for w, b in parts]
    lr_, gr = 0.0, None
    for b in range(B):
        x = ocnn.make_input(up[b], pan[b])
        z, cache = ocnn.forward(ps, x)
        g = ocnn.backward(ps, cache, z, target[b], weight=weight[b])
        lr_ += ocnn.loss(z, target[b], weight[b]) / B
        flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in g]) / B
        gr = flat if gr is None else gr + flat
    # BF16 activations and weights inside the network: the plain-FP64 bar of
    # the unweighted test
    tol = 5e-2
    assert abs(loss - lr_) <= tol * lr_, (loss, lr_)
    w_off = np.cumsum([0] + [a.size for wb in parts for a in wb])
    for k in range(len(w_off) - 1):
        a, r = grad[w_off[k]:w_off[k + 1]], gr[w_off[k]:w_off[k + 1]]
        assert np.linalg.norm(a - r) <= tol * np.linalg.norm(r) + 1e-12, k


def test_trained_diagonal_measured_against_plain_cg(cuda, c0):
    # the trained diagonal (weights/diag_cnn.npz) fits one preconditioned
    # step better than a constant diagonal, yet does not condition the Z0
    # system better: on held-out 8 x 1024^2 scenes PCG with it takes 20-27 %
    # more iterations than plain CG from the same warm start. This guards
    # that measured state: both converge, and the diagonal costs less than
    # half again the plain iterations.
    from paper_2103_09943_gb300.cnn import WarmStartNet
    path = os.path.join(WEIGHTS, "diag_cnn.npz")
    assert os.path.exists(path)
    sc, _ = c0
    cfg = sc["config"]
    dnet = WarmStartNet.load(path, device=cuda)
    wnet = WarmStartNet.load(os.path.join(WEIGHTS, "warm_cnn.npz"), device=cuda)
    args = (to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda), to_dev(sc["kernel"], cuda),
            cfg.ratio)
    common = dict(tol=1e-6, warm=2, cnn_params=wnet.params.data_ptr())
    _, _, ip = api.solve_hrms(*args, api.default_hrms_params(precond=0, **common))
    _, _, idg = api.solve_hrms(*args, api.default_hrms_params(
        precond=2, diag_params=dnet.params.data_ptr(), **common))
    assert all(s == 0 for s in ip.status + idg.status)
    assert np.mean(idg.iters) <= 1.5 * np.mean(ip.iters), (ip.iters, idg.iters)


@pytest.mark.parametrize("H,W,c,R,r", [(256, 256, 4, 4, 1), (96, 160, 2, 3, 2),
                                       (72, 48, 3, 2, 1)])
def test_jacobi_diag_matches_oracle(cuda, H, W, c, R, r):
    # diag(A) of the Z0 operator: the GPU kernel against the oracle's formula
    # (itself pinned against the dense operator's diagonal)
    from tests.gpu_util import rand_kernel
    rng = np.random.default_rng(H + W + c + R + r)
    u = rand_kernel(R, rng)
    Y = (rng.random((H, W)) * 255).astype(np.float32)
    I, mu, s = ops.pan_stats(to_dev(Y, cuda), r, 1.0)
    d = to_np(ops.jacobi_diag(to_dev(u, cuda), c, I, mu, s, r, 2e-4))
    st = oracle.pan_stats(Y, r, 1.0)
    ref = oracle.jacobi_diag(u.astype(np.float32), c, st, 2e-4)
    assert rel(d, ref) < 1e-5
    assert d.min() > 0


def test_jacobi_pcg_reaches_the_oracle(cuda):
    # PCG with P^{-1} = diag(A)^{-1} (precond = 3): the oracle's Z0 and Z at
    # the plain-form bar; its iteration count beside plain CG's, printed
    sc = synth.make_scene("c0")
    cfg = sc["config"]
    ref = oracle.solve_hrms(sc["lrms"], sc["pan"], sc["kernel"].astype(np.float64), cfg.ratio,
                            oracle.HrmsParams(tol=1e-11), threads=4)
    args = (to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda), to_dev(sc["kernel"], cuda),
            cfg.ratio)
    iters = {}
    for pc in (0, 3):
        hp = api.default_hrms_params(tol=1e-8, precond=pc, max_iter=5000)
        Z, Z0, info = api.solve_hrms(*args, hp, want_z0=True)
        assert all(st == 0 for st in info.status), (pc, info)
        for b in range(cfg.bands):
            assert rel(to_np(Z0)[b], ref["Z0"][b]) < 1e-5, (pc, b)
            assert rel(to_np(Z)[b], ref["Z"][b]) < 1e-5, (pc, b)
        iters[pc] = info.iters
    print(f"\nCG iterations to 1e-8 on the 4-band 256^2 scene: plain {iters[0]}, "
          f"Jacobi {iters[3]}")
    assert sum(iters[3]) < 2 * sum(iters[0])
