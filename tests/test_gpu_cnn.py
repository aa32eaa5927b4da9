"""GPU parity of the warm-start network's tensor-core convolution (tcgen05,
BF16 operands, FP32 accumulation) against the FP64 oracle on the same
BF16-rounded inputs and weights. The only rounding left is the FP32
accumulation order and the BF16 rounding of the output (relative 2^-9), so
the bar is 4e-3 of the output's scale."""
import numpy as np
import pytest
import torch

from oracle import cnn
from paper_2103_09943_gb300 import ops

pytestmark = pytest.mark.gpu

TOL = 4e-3


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


def _close(got, ref):
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err <= TOL * scale, (err, scale)
    assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)


@pytest.mark.parametrize("N,H,W", [(1, 8, 128), (2, 5, 256), (1, 33, 200), (1, 3, 64),
                                   (1, 70, 384)])
def test_conv32_forward_matches_oracle(cuda, N, H, W):
    rng = np.random.default_rng(N * 100 + H + W)
    x = rng.standard_normal((N, H, W, 32))
    w = rng.standard_normal((32, 32, 3, 3)) * 0.1
    b = rng.standard_normal(32) * 0.1
    xb, wb = _bf16(x), _bf16(w)
    xd = xb.to(cuda)
    wd = wb.float().to(cuda)
    bd = torch.from_numpy(b.astype(np.float32)).to(cuda)
    x64, w64 = xb.double().numpy(), wb.double().numpy()
    b64 = b.astype(np.float32).astype(np.float64)
    for mode in (0, 1):
        got = ops.cnn_conv32(xd, wd, bd, mode=mode).double().cpu().numpy()
        for n in range(N):
            ref = cnn.conv3x3(x64[n].transpose(2, 0, 1), w64, b64)
            if mode == 0:
                ref = np.maximum(ref, 0.0)
            _close(got[n].transpose(2, 0, 1), ref)


@pytest.mark.parametrize("N,H,W", [(1, 9, 128), (2, 17, 160)])
def test_conv32_adjoint_masked_matches_oracle(cuda, N, H, W):
    rng = np.random.default_rng(7 + H)
    g = rng.standard_normal((N, H, W, 32))
    m = rng.standard_normal((N, H, W, 32))
    w = rng.standard_normal((32, 32, 3, 3)) * 0.1
    gb, mb, wb = _bf16(g), _bf16(m), _bf16(w)
    got = ops.cnn_conv32(gb.to(cuda), wb.float().to(cuda), None, mode=2,
                         mask=mb.to(cuda)).double().cpu().numpy()
    g64, m64, w64 = gb.double().numpy(), mb.double().numpy(), wb.double().numpy()
    for n in range(N):
        ref = cnn.conv3x3_adjoint(g64[n].transpose(2, 0, 1), w64)
        ref = ref * (m64[n].transpose(2, 0, 1) > 0)
        _close(got[n].transpose(2, 0, 1), ref)


def _round_bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()


def _oracle_batch(params_flat, up, pan, target, bf16):
    """Loss and gradients of the batch (mean over all its pixels) by the
    oracle, per band; with bf16, the 32 -> 32 weights and the hidden
    activations and gradients are rounded where the GPU stores them as BF16."""
    from paper_2103_09943_gb300.cnn import split_params
    ps = [(w.astype(np.float64), b.astype(np.float64)) for w, b in split_params(params_flat)]
    ra = rg = None
    if bf16:
        ps = [(_round_bf16(w) if 1 <= l <= 4 else w, b) for l, (w, b) in enumerate(ps)]
        ra = rg = _round_bf16
    B = up.shape[0]
    zs, loss, grads = [], 0.0, None
    for b in range(B):
        x = cnn.make_input(up[b], pan[b])
        z, cache = cnn.forward(ps, x, round_act=ra)
        g = cnn.backward(ps, cache, z, target[b], round_grad=rg)
        zs.append(z)
        loss += cnn.loss(z, target[b]) / B
        flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in g]) / B
        grads = flat if grads is None else grads + flat
    return np.stack(zs), loss, grads


def test_network_forward_and_gradients_match_oracle(cuda):
    from paper_2103_09943_gb300.cnn import WarmStartNet, init_params, split_params
    rng = np.random.default_rng(21)
    B, H, W = 2, 24, 40
    p = init_params(5)
    # a last layer and biases far from their initial values, so that every
    # gradient is exercised
    parts = split_params(p)
    parts[-1][0][...] *= 10.0
    for _, b in parts:
        b[...] = rng.standard_normal(b.shape) * 0.05
    up = (rng.random((B, H, W)) * 255).astype(np.float32)
    pan = (rng.random((B, H, W)) * 255).astype(np.float32)
    target = (up + rng.standard_normal((B, H, W)) * 20).astype(np.float32)
    net = WarmStartNet(params=p, device=cuda)
    dev = lambda a: torch.from_numpy(a).to(cuda)
    z = net.forward(dev(up), dev(pan), check=True).double().cpu().numpy()
    loss = net.loss_grad(dev(up), dev(pan), dev(target))
    grad = net.grad.double().cpu().numpy()
    w_off = np.cumsum([0] + [a.size for wb in parts for a in wb])
    for bf16, tol in ((False, 5e-2), (True, 1e-2)):
        zr, lr_, gr = _oracle_batch(p, up, pan, target, bf16)
        assert np.linalg.norm((z - up) - (zr - up)) <= tol * np.linalg.norm(zr - up), bf16
        assert abs(loss - lr_) <= tol * lr_, (bf16, loss, lr_)
        for k in range(len(w_off) - 1):
            a, r = grad[w_off[k]:w_off[k + 1]], gr[w_off[k]:w_off[k + 1]]
            assert np.linalg.norm(a - r) <= tol * np.linalg.norm(r) + 1e-12, (bf16, k)


def test_adam_steps_lower_the_loss(cuda):
    from paper_2103_09943_gb300.cnn import WarmStartNet
    rng = np.random.default_rng(3)
    B, H, W = 2, 32, 64
    up = torch.from_numpy((rng.random((B, H, W)) * 255).astype(np.float32)).to(cuda)
    pan = torch.from_numpy((rng.random((H, W)) * 255).astype(np.float32)).to(cuda)
    target = up + 10.0 * (pan[None] / 255.0 - 0.5)
    net = WarmStartNet(seed=1, device=cuda)
    first = net.loss_grad(up, pan, target)
    for _ in range(30):
        net.loss_grad(up, pan, target)
        net.adam(lr=2e-3)
    assert net.loss_grad(up, pan, target) < 0.5 * first


@pytest.mark.parametrize("B,H,W,shared_pan", [(1, 70, 300, True), (2, 33, 132, False)])
def test_fused_forward_matches_oracle(cuda, B, H, W, shared_pan):
    # several 126-pixel strips (the last one partial) and row chunks: the
    # first layer computed inside the first tensor-core layer, the last one
    # in the epilogue of the fourth
    from paper_2103_09943_gb300.cnn import WarmStartNet, init_params, split_params
    rng = np.random.default_rng(B + H + W)
    p = init_params(9)
    parts = split_params(p)
    parts[-1][0][...] *= 10.0
    up = (rng.random((B, H, W)) * 255).astype(np.float32)
    pan = (rng.random((H, W) if shared_pan else (B, H, W)) * 255).astype(np.float32)
    net = WarmStartNet(params=p, device=cuda)
    z = net.forward(torch.from_numpy(up).to(cuda), torch.from_numpy(pan).to(cuda),
                    check=True).double().cpu().numpy()
    pans = np.broadcast_to(pan, (B, H, W)) if shared_pan else pan
    for bf16, tol in ((False, 5e-2), (True, 1e-2)):
        zr, _, _ = _oracle_batch(p, up, pans, up, bf16)
        assert np.linalg.norm((z - up) - (zr - up)) <= tol * np.linalg.norm(zr - up), bf16
