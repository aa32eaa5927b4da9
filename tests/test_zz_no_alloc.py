"""The allocation-free entry point (ps_op_kernel_normal_eq_noalloc) gives the
results of the workspace entry point it mirrors.

It serves callers that may not allocate device memory on their call path; its
scratch is a fixed array owned by the library and shared by all calls. This
file is collected last on purpose, and its checks stand alone: two calls in a
row on different inputs, each against ps_op_kernel_normal_eq.
"""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def _inputs(seed, N, H, c):
    rng = np.random.default_rng(seed)
    Y = (rng.random((H, H)) * 255).astype(np.float32)
    X = (rng.random((N, H // c, H // c)) * 255).astype(np.float32)
    om = rng.dirichlet(np.ones(N)).astype(np.float32)
    return X, Y, om


@pytest.mark.parametrize("N,H,c,R", [(4, 256, 4, 4), (8, 1024, 4, 8), (3, 96, 2, 5)])
def test_noalloc_matches_workspace_entry_point(cuda, N, H, c, R):
    from paper_2103_09943_gb300 import ops
    for call in range(2):
        X, Y, om = _inputs(100 * call + H + R, N, H, c)
        gx, gy, go = to_dev(X, cuda), to_dev(Y, cuda), to_dev(om, cuda)
        ref_e, ref_f = ops.kernel_normal_eq(gx, gy, go, c, R)
        e, f = ops.kernel_normal_eq_noalloc(gx, gy, go, c, R)
        assert rel(to_np(e), to_np(ref_e)) < 1e-12
        assert rel(to_np(f), to_np(ref_f)) < 1e-12


def test_noalloc_matches_the_oracle_on_a_non_square_grid(cuda):
    # E^T E and E^T f by their plain definition (the FP64 oracle), on a
    # 96 x 160 PAN at ratio 2: rows and columns of the LR grid differ, so a
    # transposed index would show.
    import oracle
    from paper_2103_09943_gb300 import ops
    N, H, W, c, R = 3, 96, 160, 2, 5
    rng = np.random.default_rng(7)
    Y = (rng.random((H, W)) * 255).astype(np.float32)
    X = (rng.random((N, H // c, W // c)) * 255).astype(np.float32)
    om = rng.dirichlet(np.ones(N)).astype(np.float32)
    f = np.tensordot(om.astype(np.float64), X.astype(np.float64), axes=1)
    ref_e, ref_f = oracle.kernel_normal_eq(Y, f, c, R)
    gx, gy, go = to_dev(X, cuda), to_dev(Y, cuda), to_dev(om, cuda)
    for _ in range(2):
        e, g = ops.kernel_normal_eq_noalloc(gx, gy, go, c, R)
        # double-float accumulation of exact FP32 products; f formed in FP32
        assert rel(to_np(e), ref_e) < 1e-12
        assert rel(to_np(g), ref_f) < 1e-6


def test_noalloc_rejects_sizes_beyond_its_array(cuda):
    from paper_2103_09943_gb300 import _lib
    lib = _lib.load()
    fake = ctypes.c_void_p(0x1000)
    # LR grid 2048 x 2048: 16 MiB of f alone, more than the 4 MiB array
    st = lib.ps_op_kernel_normal_eq_noalloc(fake, fake, fake, 8, 8192, 8192, 4, 8, fake, fake,
                                            None)
    assert st == 8
