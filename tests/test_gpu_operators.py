"""GPU parity of the image-domain operators against the FP64 oracle, through
the operator-level C-ABI (include/ps_ops.h), on sizes that span several
tiles with ragged tails, plus the degenerate kernel R = 0 and the largest
kernel and window supported."""
import numpy as np
import pytest

import oracle
from paper_2103_09943_gb300 import ops
from tests.gpu_util import rand_kernel, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

# (H, W, c, R): LLP tiles are 32 x 32, LR tiles 8 x 32 sites -> ragged tails
SIZES = [(96, 96, 4, 3), (144, 96, 4, 8), (64, 128, 2, 2), (120, 72, 3, 4),
         (40, 24, 4, 0), (192, 160, 4, 16)]
FP32_TOL = 2e-6


@pytest.mark.parametrize("H,W,c,R", SIZES)
def test_blur_decimate_and_adjoint(cuda, H, W, c, R):
    rng = np.random.default_rng(H * 7 + W + R)
    N = 3
    z = rng.random((N, H, W)) * 255
    v = rng.random((N, H // c, W // c)) * 255
    u = rand_kernel(R, rng)
    gz, gv, gu = to_dev(z, cuda), to_dev(v, cuda), to_dev(u, cuda)
    db = to_np(ops.blur_decimate(gz, gu, c))
    ad = to_np(ops.blur_decimate_adj(gv, gu, c))
    u32 = u.astype(np.float32).astype(np.float64)
    for b in range(N):
        zb = z[b].astype(np.float32).astype(np.float64)
        vb = v[b].astype(np.float32).astype(np.float64)
        assert rel(db[b], oracle.blur_decimate(zb, u32, c)) < FP32_TOL
        assert rel(ad[b], oracle.blur_decimate_adj(vb, u32, c)) < FP32_TOL


@pytest.mark.parametrize("r", [1, 2, 4])
@pytest.mark.parametrize("H,W", [(96, 96), (120, 72)])
def test_pan_stats(cuda, H, W, r):
    rng = np.random.default_rng(r + H)
    Y = (rng.random((H, W)) * 255).astype(np.float32)
    eps = 1.0
    I, mu, s = (to_np(t) for t in ops.pan_stats(to_dev(Y, cuda), r, eps))
    st = oracle.pan_stats(Y.astype(np.float64), r, eps)
    assert rel(I, st.I) < 1e-7
    assert rel(mu, st.mu) < 1e-7
    assert rel(s, st.s) < 1e-6


def _stats32(Y, r, eps):
    st = oracle.pan_stats(Y, r, eps)
    I32, mu32, s32 = (a.astype(np.float32) for a in (st.I, st.mu, st.s))
    st64 = oracle.PanStats(I32.astype(np.float64), mu32.astype(np.float64), st.var,
                           s32.astype(np.float64), r, eps)
    return st64, (I32, mu32, s32)


@pytest.mark.parametrize("H,W,c,R,r", [(96, 96, 4, 3, 1), (144, 96, 4, 8, 2),
                                       (120, 72, 3, 4, 1), (64, 64, 2, 1, 4)])
def test_apply_z0_operator(cuda, H, W, c, R, r):
    rng = np.random.default_rng(H + 10 * r)
    N, eps, lam = 2, 1.0, 2e-4
    Y = (rng.random((H, W)) * 255).astype(np.float64)
    st, (I, mu, s) = _stats32(Y, r, eps)
    u = rand_kernel(R, rng).astype(np.float32)
    z = (rng.random((N, H, W)) * 255).astype(np.float32)
    out = to_np(ops.apply_z0(to_dev(z, cuda), to_dev(u, cuda), c, to_dev(I, cuda),
                             to_dev(mu, cuda), to_dev(s, cuda), r, lam))
    for b in range(N):
        ref = oracle.apply_z0_system(z[b].astype(np.float64), u.astype(np.float64), c, st, lam)
        assert rel(out[b], ref) < 1e-5
    # the prior part alone (lam large, so it dominates), checks L M L
    lam2 = 1.0
    out = to_np(ops.apply_z0(to_dev(z, cuda), to_dev(u, cuda), c, to_dev(I, cuda),
                             to_dev(mu, cuda), to_dev(s, cuda), r, lam2))
    ref = oracle.apply_z0_system(z[0].astype(np.float64), u.astype(np.float64), c, st, lam2)
    assert rel(out[0], ref) < 1e-5


@pytest.mark.parametrize("H,W,r", [(96, 96, 1), (144, 96, 2), (120, 72, 3)])
def test_guided_filter(cuda, H, W, r):
    rng = np.random.default_rng(H + r)
    Y = rng.random((H, W)) * 255
    st, (I, mu, s) = _stats32(Y, r, 1.0)
    q = (rng.standard_normal((3, H, W)) * 40).astype(np.float32)
    out = to_np(ops.guided_filter(to_dev(q, cuda), to_dev(I, cuda), to_dev(mu, cuda),
                                  to_dev(s, cuda), r))
    for b in range(3):
        ref = oracle.guided_filter(q[b].astype(np.float64), st)
        assert rel(out[b], ref) < 1e-5


def test_many_bands_small_image(cuda):
    # the largest band count on a small torus
    rng = np.random.default_rng(0)
    N, H, W, c, R = 64, 32, 32, 4, 2
    z = (rng.random((N, H, W)) * 255).astype(np.float32)
    u = rand_kernel(R, rng).astype(np.float32)
    db = to_np(ops.blur_decimate(to_dev(z, cuda), to_dev(u, cuda), c))
    for b in (0, 31, 63):
        assert rel(db[b], oracle.blur_decimate(z[b].astype(np.float64),
                                               u.astype(np.float64), c)) < FP32_TOL
