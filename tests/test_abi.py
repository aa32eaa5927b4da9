"""The C-ABI library loads and exports every entry point declared in
include/*.h; host-side parts (defaults, workspace sizes, argument checks that
return before any launch) behave as documented. No GPU needed."""
import ctypes
import os
import re
import subprocess

import pytest

from tests.golden.load import paper_parameters

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib
    importlib.import_module("paper_2103_09943_gb300.build").build()
    from paper_2103_09943_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(ps_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    from paper_2103_09943_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 15
    so = os.path.join(ROOT, "paper_2103_09943_gb300", "_build", "libps.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (ps_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the Python binding declares exactly the header's entry points
    assert sorted(_lib.SIGNATURES) == names


def test_defaults_are_the_paper_values(lib):
    from paper_2103_09943_gb300._lib import HrmsParams, KernelParams
    p = paper_parameters()
    kp = KernelParams()
    lib.ps_default_kernel_params(ctypes.byref(kp))
    for name in ("lambda_omega", "alpha1", "alpha2", "mu1", "mu2", "mu3", "rho", "t_max"):
        assert getattr(kp, name) == pytest.approx(p[name], rel=1e-6), name
    assert kp.th == pytest.approx(p["th"], rel=1e-6)
    hp = HrmsParams()
    lib.ps_default_hrms_params(ctypes.byref(hp))
    assert hp.lambda_ == pytest.approx(p["lambda"], rel=1e-6)
    assert hp.r == p["r"]
    # the preconditioned CG (an extension) is on by default, gamma = 4
    assert hp.precond == 1 and hp.precond_gamma == pytest.approx(4.0)


def test_workspace_size(lib):
    assert lib.ps_workspace_size(4, 256, 256, 4, 4, None) > 4 * 256 * 256 * 4 * 4
    assert lib.ps_workspace_size(8, 1024, 1024, 4, 8, None) > 0
    assert lib.ps_workspace_size(4, 256, 250, 4, 4, None) == 0      # W % c
    assert lib.ps_workspace_size(4, 256, 256, 1, 4, None) == 0      # ratio < 2
    assert lib.ps_workspace_size(0, 256, 256, 4, 4, None) == 0      # no bands
    assert lib.ps_workspace_size(4, 16, 16, 4, 9, None) == 0       # kernel > image


def test_status_strings(lib):
    for s in range(10):
        assert lib.ps_status_string(s) != b"unknown status"
    assert lib.ps_status_string(0) == b"ok"


def test_argument_errors_return_before_launch(lib):
    from paper_2103_09943_gb300._lib import HrmsParams, KernelParams
    hp = HrmsParams()
    lib.ps_default_hrms_params(ctypes.byref(hp))
    kp = KernelParams()
    lib.ps_default_kernel_params(ctypes.byref(kp))
    fake = ctypes.c_void_p(0x1000)
    # shape: H not a multiple of the ratio
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 250, 256, 4, 4, ctypes.byref(hp), None, fake,
                           None, None, fake, 1 << 30, None)
    assert st == 2
    # FFT sizes must be 2^a 3^b
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 260, 260, 4, 4, ctypes.byref(hp), None, fake,
                           None, None, fake, 1 << 30, None)
    assert st == 8
    # bad parameter
    bad = HrmsParams.from_buffer_copy(hp)
    bad.eps = 0.0
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bad), None, fake,
                           None, None, fake, 1 << 30, None)
    assert st == 1
    # null output
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(hp), None, None,
                           None, None, fake, 1 << 30, None)
    assert st == 1
    # workspace too small / misaligned
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(hp), None, fake,
                           None, None, fake, 1024, None)
    assert st == 4
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(hp), None, fake,
                           None, None, ctypes.c_void_p(0x1010), 1 << 30, None)
    assert st == 4
    # preconditioner selector and weight
    bad = HrmsParams.from_buffer_copy(hp)
    bad.precond = 2
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bad), None, fake,
                           None, None, fake, 1 << 30, None)
    assert st == 1
    bad = HrmsParams.from_buffer_copy(hp)
    bad.precond_gamma = 0.0
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bad), None, fake,
                           None, None, fake, 1 << 30, None)
    assert st == 1
    # the diagonal preconditioner: a selector in 0..3, a 16-byte aligned
    # diagonal, and room for the diagonal network when it supplies s
    bad = HrmsParams.from_buffer_copy(hp)
    bad.precond = 4
    bad.precond_diag = 0x1000
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bad), None, fake,
                           None, None, fake, 1 << 30, None)
    assert st == 1
    bad.precond = 2
    bad.precond_diag = 0x1004
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bad), None, fake,
                           None, None, fake, 1 << 30, None)
    assert st == 1
    bad.precond_diag = None
    bad.diag_params = 0x1000
    need = lib.ps_workspace_size(4, 256, 256, 4, 4, ctypes.byref(bad))
    assert need > lib.ps_workspace_size(4, 256, 256, 4, 4, ctypes.byref(hp))
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bad), None, fake,
                           None, None, fake, lib.ps_workspace_size(4, 256, 256, 4, 4, None), None)
    assert st == 4                                                  # no room for the network
    st = lib.ps_op_precond(fake, 2, 96, 96, 4, fake, 3, ctypes.c_float(-1.0), fake, fake,
                           1 << 30, None)
    assert st == 1
    # alternative priors: a valid id, and the plain CG
    bad = HrmsParams.from_buffer_copy(hp)
    bad.prior = 5
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bad), None, fake,
                           None, None, fake, 1 << 30, None)
    assert st == 1
    bad.prior = 4
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bad), None, fake,
                           None, None, fake, 1 << 30, None)
    assert st == 1                                                  # precond with a prior
    bad.precond = 0
    need = lib.ps_workspace_size(4, 256, 256, 4, 4, ctypes.byref(bad))
    assert need > lib.ps_workspace_size(4, 256, 256, 4, 4, ctypes.byref(hp))
    st = lib.ps_solve_hrms(fake, fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bad), None, fake,
                           None, None, fake, need - 1024, None)
    assert st == 4                                                  # its scratch is missing
    st = lib.ps_op_precond(fake, 2, 100, 100, 4, fake, 3, ctypes.c_float(1e-3), fake, fake,
                           1 << 30, None)
    assert st == 8                                                  # not 2^a 3^b
    bk = KernelParams.from_buffer_copy(kp)
    bk.mu3 = -1.0
    st = lib.ps_estimate_kernel(fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bk), None, fake,
                                None, None, fake, 1 << 30, None)
    assert st == 1
    st = lib.ps_pansharpen(fake, fake, 4, 256, 256, 4, 17, ctypes.byref(kp), ctypes.byref(hp),
                           fake, None, None, None, fake, 1 << 30, None)
    assert st == 1                                                  # R > 16
    # the X' mask of Eq. objective1 may select only bands that exist
    bk = KernelParams.from_buffer_copy(kp)
    bk.band_mask = 1 << 4                                           # band 4 of 4
    st = lib.ps_estimate_kernel(fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bk), None, fake,
                                None, None, fake, 1 << 30, None)
    assert st == 1
    st = lib.ps_pansharpen(fake, fake, 4, 256, 256, 4, 4, ctypes.byref(bk), ctypes.byref(hp),
                           fake, None, None, None, fake, 1 << 30, None)
    assert st == 1


def test_noalloc_shape_limits_are_its_twins(lib):
    # The allocation-free entry point applies the workspace entry point's
    # size limits (same status codes) before its own scratch limit.
    fake = ctypes.c_void_p(0x1000)
    cases = [((4, 96, 98, 2, 4), 8),      # W % 4: the lag kernels' float4 rows
             ((4, 98, 96, 4, 4), 2),      # H % ratio
             ((4, 16384, 96, 4, 4), 8),   # beyond the largest image side
             ((4, 96, 96, 4, 17), 1),     # R > 16
             ((0, 96, 96, 4, 4), 1)]      # no bands
    for (N, H, W, c, R), want in cases:
        twin = lib.ps_op_kernel_normal_eq(fake, fake, fake, N, H, W, c, R, fake, fake, fake,
                                          1 << 30, None)
        st = lib.ps_op_kernel_normal_eq_noalloc(fake, fake, fake, N, H, W, c, R, fake, fake,
                                                None)
        assert st == twin == want, ((N, H, W, c, R), st, twin)


def test_batched_argument_errors_return_before_launch(lib):
    from paper_2103_09943_gb300._lib import HrmsParams, KernelParams, Scene
    hp = HrmsParams()
    lib.ps_default_hrms_params(ctypes.byref(hp))
    kp = KernelParams()
    lib.ps_default_kernel_params(ctypes.byref(kp))
    f = 0x1000
    arr = (Scene * 3)(Scene(f, f, f, f, 4, 512, 512, 4, 4), Scene(f, f, f, f, 8, 768, 768, 4, 8),
                      Scene(f, f, f, f, 4, 1536, 1536, 4, 6))
    need = lib.ps_batch_workspace_size(arr, 3, ctypes.byref(hp))
    singles = sum(lib.ps_workspace_size(s.N, s.H, s.W, s.ratio, s.R, ctypes.byref(hp))
                  for s in arr)
    assert need >= singles + 4 * 8
    ws = ctypes.c_void_p(0x100000)
    # workspace too small, misaligned
    assert lib.ps_pansharpen_batched(arr, 3, ctypes.byref(kp), ctypes.byref(hp), None, None,
                                     ws, need - 1, None) == 4
    assert lib.ps_pansharpen_batched(arr, 3, ctypes.byref(kp), ctypes.byref(hp), None, None,
                                     ctypes.c_void_p(0x100010), need, None) == 4
    # the batch is one graph: no host-driven loop
    bad = HrmsParams.from_buffer_copy(hp)
    bad.host_loop = 1
    assert lib.ps_pansharpen_batched(arr, 3, ctypes.byref(kp), ctypes.byref(bad), None, None,
                                     ws, need, None) == 1
    # one diagonal array cannot serve every scene
    bad = HrmsParams.from_buffer_copy(hp)
    bad.precond = 2
    bad.precond_diag = 0x1000
    assert lib.ps_pansharpen_batched(arr, 3, ctypes.byref(kp), ctypes.byref(bad), None, None,
                                     ws, need, None) == 1
    # empty batch, one bad scene among good ones
    assert lib.ps_pansharpen_batched(arr, 0, ctypes.byref(kp), ctypes.byref(hp), None, None,
                                     ws, need, None) == 1
    arr[1].H = 770
    assert lib.ps_batch_workspace_size(arr, 3, ctypes.byref(hp)) == 0
    assert lib.ps_pansharpen_batched(arr, 3, ctypes.byref(kp), ctypes.byref(hp), None, None,
                                     ws, need, None) == 2
    arr[1].H = 768
    arr[2].kernel = None
    assert lib.ps_pansharpen_batched(arr, 3, ctypes.byref(kp), ctypes.byref(hp), None, None,
                                     ws, need, None) == 1
    arr[2].kernel = f
    # a scene's X' mask selects bands that exist in that scene
    arr[0].band_mask = 1 << 5                                       # scene 0 has 4 bands
    assert lib.ps_pansharpen_batched(arr, 3, ctypes.byref(kp), ctypes.byref(hp), None, None,
                                     ws, need, None) == 1
    arr[0].band_mask = 0
    bk = KernelParams.from_buffer_copy(kp)
    bk.band_mask = 1 << 6                                           # fine for the 8-band scene only
    assert lib.ps_pansharpen_batched(arr, 3, ctypes.byref(bk), ctypes.byref(hp), None, None,
                                     ws, need, None) == 1


def test_tuning_arguments(lib):
    from paper_2103_09943_gb300._lib import Tuning
    t = Tuning()
    t.split = 3
    assert lib.ps_set_tuning(4, 256, 256, 4, 1, ctypes.byref(t)) == 1
    t.split, t.llp_bands = 2, 3
    assert lib.ps_set_tuning(4, 256, 256, 4, 1, ctypes.byref(t)) == 1
    t.llp_bands, t.llp_pf = 2, 5
    assert lib.ps_set_tuning(4, 256, 256, 4, 1, ctypes.byref(t)) == 1
    t.llp_pf, t.llp_form = 4, 3
    assert lib.ps_set_tuning(4, 256, 256, 4, 1, ctypes.byref(t)) == 1
    t.llp_form = 4                                 # lean walks: one band per CTA only
    assert lib.ps_set_tuning(4, 256, 256, 4, 1, ctypes.byref(t)) == 1
    t.llp_bands = 1
    assert lib.ps_set_tuning(4, 256, 256, 4, 2, ctypes.byref(t)) == 1   # and r = 1 only
    t.llp_rows = 66                                # the general walk's length
    assert lib.ps_set_tuning(4, 256, 256, 4, 1, ctypes.byref(t)) == 1
    t.llp_rows, t.llp_form, t.llp_pf = 0, 2, 3     # lean walks: 2 or 4 rows ahead
    assert lib.ps_set_tuning(4, 256, 256, 4, 1, ctypes.byref(t)) == 1
    t.llp_form, t.llp_pf, t.llp_bands = 0, 4, 2
    assert lib.ps_set_tuning(4, 250, 256, 4, 1, ctypes.byref(t)) == 2   # H % ratio
    assert lib.ps_set_tuning(4, 256, 256, 4, 1, None) == 1

