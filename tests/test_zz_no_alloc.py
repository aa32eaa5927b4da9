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


def test_noalloc_rejects_sizes_beyond_its_array(cuda):
    from paper_2103_09943_gb300 import _lib
    lib = _lib.load()
    fake = ctypes.c_void_p(0x1000)
    # LR grid 2048 x 2048: 16 MiB of f alone, more than the 4 MiB array
    st = lib.ps_op_kernel_normal_eq_noalloc(fake, fake, fake, 8, 8192, 8192, 4, 8, fake, fake,
                                            None)
    assert st == 8
