"""GPU parity of Algorithm 2 (the per-band HRMS solve) against the FP64
oracle: the Z step alone, then Z0 and Z of ps_solve_hrms, on the 4-band
256 x 256 scene and on smaller ragged and odd-band cases; warm start;
device-side statuses."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2103_09943_gb300 import api, ops
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu

# Plain FP32 form: FP32 vectors and operators, FP64 reductions (and the FP64
# forward FFT of the Z step). The CG stops at a recursive relative residual of
# 1e-8; the bar against the oracle is rel-L2 <= 1e-5 per band.
PLAIN_TOL = 1e-5
CG_TOL = 1e-8


def _scene(cfg, **kw):
    return synth.make_scene(replace(cfg, **kw) if kw else cfg)


def test_zstep_given_oracle_z0(cuda):
    sc = _scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    c, r, lam = cfg.ratio, 1, 2e-4
    u = sc["kernel"].astype(np.float64)
    hp = oracle.HrmsParams(tol=1e-11)
    st = oracle.pan_stats(sc["pan"], r, hp.eps)
    I, mu, s = (a.astype(np.float32) for a in (st.I, st.mu, st.s))
    for exact in (False, True):
        hp.exact_weight = exact
        for b in (0, 3):
            ob = oracle.solve_band(sc["lrms"][b], u, c, st, hp)
            z0 = ob["Z0"].astype(np.float32)
            gz = ops.zstep(to_dev(sc["lrms"][b:b + 1], cuda), to_dev(z0[None], cuda),
                           to_dev(sc["kernel"], cuda), c, to_dev(I, cuda), to_dev(mu, cuda),
                           to_dev(s, cuda), r, lam, exact_weight=exact)
            assert rel(to_np(gz)[0], ob["Z"]) < PLAIN_TOL


@pytest.fixture(scope="module")
def c0_oracle():
    sc = _scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    ref = oracle.solve_hrms(sc["lrms"], sc["pan"], sc["kernel"].astype(np.float64),
                            cfg.ratio, oracle.HrmsParams(tol=1e-11), threads=4)
    return sc, ref


def test_solve_hrms_c0_plain_fp32(cuda, c0_oracle):
    sc, ref = c0_oracle
    cfg = sc["config"]
    hp = api.default_hrms_params(tol=CG_TOL, max_iter=5000)
    Z, Z0, info = api.solve_hrms(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                 to_dev(sc["kernel"], cuda), cfg.ratio, hp, want_z0=True)
    Z, Z0 = to_np(Z), to_np(Z0)
    assert all(s == 0 for s in info.status), info
    for b in range(cfg.bands):
        assert rel(Z0[b], ref["Z0"][b]) < PLAIN_TOL, (b, info)
        assert rel(Z[b], ref["Z"][b]) < PLAIN_TOL, (b, info)


def test_solve_hrms_default_tolerance_meets_1e3(cuda, c0_oracle):
    sc, ref = c0_oracle
    cfg = sc["config"]
    Z, _, info = api.solve_hrms(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                to_dev(sc["kernel"], cuda), cfg.ratio)
    Z = to_np(Z)
    for b in range(cfg.bands):
        assert rel(Z[b], ref["Z"][b]) < 1e-3


def test_warm_start_from_solution(cuda, c0_oracle):
    sc, ref = c0_oracle
    cfg = sc["config"]
    hp = api.default_hrms_params(tol=CG_TOL)
    zi = to_dev(ref["Z0"], cuda)
    Z, Z0, info = api.solve_hrms(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                 to_dev(sc["kernel"], cuda), cfg.ratio, hp, z_init=zi,
                                 want_z0=True)
    assert max(info.iters) < 150, info
    assert max(rel(to_np(Z0)[b], ref["Z0"][b]) for b in range(cfg.bands)) < PLAIN_TOL


@pytest.mark.parametrize("N,H,W,c,R,r", [(3, 144, 96, 4, 5, 1), (1, 96, 96, 2, 3, 2),
                                         (2, 72, 108, 3, 4, 1)])
def test_solve_hrms_ragged_and_odd(cuda, N, H, W, c, R, r):
    base = synth.CONFIGS["c0"]
    sc = _scene(base, bands=N, H=H, W=W, ratio=c, R=R, shapes=15, seed=40 + N)
    u = sc["kernel"].astype(np.float64)
    ref = oracle.solve_hrms(sc["lrms"], sc["pan"], u, c, oracle.HrmsParams(r=r, tol=1e-11),
                            threads=3)
    hp = api.default_hrms_params(tol=CG_TOL, r=r, max_iter=5000)
    Z, Z0, info = api.solve_hrms(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                 to_dev(sc["kernel"], cuda), c, hp, want_z0=True)
    Z, Z0 = to_np(Z), to_np(Z0)
    for b in range(N):
        assert rel(Z0[b], ref["Z0"][b]) < PLAIN_TOL, (b, info)
        assert rel(Z[b], ref["Z"][b]) < PLAIN_TOL, (b, info)


def test_status_not_converged_and_zero_band(cuda):
    sc = _scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    X = sc["lrms"].copy()
    X[1] = 0.0                                  # b = 0: done at once, Z = 0
    hp = api.default_hrms_params(tol=1e-12, max_iter=3)
    Z, _, info = api.solve_hrms(to_dev(X, cuda), to_dev(sc["pan"], cuda),
                                to_dev(sc["kernel"], cuda), cfg.ratio, hp)
    assert info.status[0] == 5 and info.iters[0] == 3
    assert info.status[1] == 0 and info.iters[1] == 0
    # band 1 shares its complex FFT image with band 0: only FP32 round-off of
    # band 0 can reach it
    Zn = to_np(Z)
    assert np.max(np.abs(Zn[1])) < 1e-5 * np.max(np.abs(Zn[0]))


def test_status_nonfinite_input(cuda):
    sc = _scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    X = sc["lrms"].copy()
    X[2, 5, 7] = np.nan
    Z, _, info = api.solve_hrms(to_dev(X, cuda), to_dev(sc["pan"], cuda),
                                to_dev(sc["kernel"], cuda), cfg.ratio)
    assert info.status[2] == 6
    assert info.status[0] == 0


def test_host_loop_matches_device_loop(cuda, c0_oracle):
    sc, ref = c0_oracle
    cfg = sc["config"]
    args = (to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda), to_dev(sc["kernel"], cuda),
            cfg.ratio)
    Zg, _, ig = api.solve_hrms(*args, api.default_hrms_params(tol=1e-7))
    Zh, _, ih = api.solve_hrms(*args, api.default_hrms_params(tol=1e-7, host_loop=1))
    assert ig.iters == ih.iters
    assert rel(to_np(Zh), to_np(Zg)) < 1e-6


def test_paper_stop_rule_matches_oracle(cuda):
    # Sec. IV-F: the paper's CG for Z0 runs from zeros and stops when the
    # relative change of the iterate (Frobenius norm) falls below 5e-5. The
    # GPU stops at the oracle's iteration and lands on its iterate (measured:
    # equal counts, rel-L2 6e-6).
    sc = _scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    ref = oracle.solve_hrms(sc["lrms"], sc["pan"], sc["kernel"].astype(np.float64), cfg.ratio,
                            oracle.HrmsParams(tol=5e-5, stop_rule=1), threads=4)
    hp = api.default_hrms_params(tol=5e-5, stop_rule=1, precond=0, max_iter=5000)
    Z, Z0, info = api.solve_hrms(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                 to_dev(sc["kernel"], cuda), cfg.ratio, hp, want_z0=True)
    Z, Z0 = to_np(Z), to_np(Z0)
    assert all(s == 0 for s in info.status), info
    for b in range(cfg.bands):
        assert abs(info.iters[b] - ref["bands"][b]["iters_z0"]) <= 2, (b, info.iters)
        assert rel(Z0[b], ref["Z0"][b]) < 1e-4, b
        assert rel(Z[b], ref["Z"][b]) < 1e-4, b


def test_paper_stop_rule_with_preconditioner_stops_earlier(cuda):
    # the rule is the same with the preconditioner; it stops much sooner and
    # (measured) closer to the exact solution
    sc = _scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    args = (to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda), to_dev(sc["kernel"], cuda),
            cfg.ratio)
    it = {}
    for pc in (0, 1):
        hp = api.default_hrms_params(tol=5e-5, stop_rule=1, precond=pc, max_iter=5000)
        _, _, info = api.solve_hrms(*args, hp)
        assert all(s == 0 for s in info.status), info
        it[pc] = info.iters
    assert max(it[1]) * 2 < min(it[0]), it


def test_zstep_fp32_within_its_bound(cuda, c0_oracle):
    # the all-FP32 Z step (the preconditioner's register FFTs and group
    # solve): the forward spectrum's rounding, amplified by the Z-step
    # operator's condition number (~200), costs ~6e-6 rel-L2 (numpy
    # experiment); the bar leaves a factor of five, far inside the 1e-3 of
    # the mixed-precision form
    sc, ref = c0_oracle
    cfg = sc["config"]
    args = (to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda), to_dev(sc["kernel"], cuda),
            cfg.ratio)
    out = {}
    for fp32 in (0, 1):
        hp = api.default_hrms_params(tol=CG_TOL, max_iter=5000, zstep_fp32=fp32)
        Z, Z0, info = api.solve_hrms(*args, hp, want_z0=True)
        out[fp32] = (to_np(Z), to_np(Z0), info.iters)
    assert out[0][2] == out[1][2]
    for b in range(cfg.bands):
        assert rel(out[1][1][b], out[0][1][b]) < 1e-6   # same Z0
        assert rel(out[1][0][b], out[0][0][b]) < 3e-5
        assert rel(out[1][0][b], ref["Z"][b]) < 3e-5


def test_sticky_status_after_calls_without_info(cuda):
    # Calls without h_info return before their work runs; ps_sync_status waits
    # for the stream and reports (then clears) the first device-detected
    # status of the calls since the last read: here a band stopped on a
    # non-finite value, then nothing.
    sc = _scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    Xd, Yd = to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda)
    Kd = to_dev(sc["kernel"], cuda)
    assert api.sync_status() in (0, 5, 6, 7)     # whatever earlier tests left
    api.solve_hrms(Xd, Yd, Kd, cfg.ratio, info=False)
    assert api.sync_status() == 0
    X = sc["lrms"].copy()
    X[2, 5, 7] = np.nan
    api.solve_hrms(to_dev(X, cuda), Yd, Kd, cfg.ratio, info=False)
    api.solve_hrms(Xd, Yd, Kd, cfg.ratio, api.default_hrms_params(tol=1e-12, max_iter=3),
                   info=False)
    assert api.sync_status() == 6                 # the first one recorded
    assert api.sync_status() == 0                 # and cleared
    api.solve_hrms(Xd, Yd, Kd, cfg.ratio, api.default_hrms_params(tol=1e-12, max_iter=3),
                   info=False)
    assert api.sync_status() == 5


def test_band_solve_times(cuda):
    # Per-band device time of the Z0 solve: positive, within the call's own
    # time, and longer for a band that ran more iterations in the same loop.
    sc = _scene(synth.CONFIGS["c0"])
    cfg = sc["config"]
    X = sc["lrms"].copy()
    X[1] = 0.0                                  # stops before its first iteration
    hp = api.default_hrms_params(precond=0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    _, _, info = api.solve_hrms(to_dev(X, cuda), to_dev(sc["pan"], cuda),
                                to_dev(sc["kernel"], cuda), cfg.ratio, hp)
    b.record()
    torch.cuda.synchronize()
    total = a.elapsed_time(b)
    ms = info.ms
    assert all(0.0 < t <= total * 1.05 for t in ms), (ms, total)
    assert ms[1] < min(ms[0], ms[2], ms[3]), ms
    assert info.iters[1] == 0 and min(info.iters[0], info.iters[2], info.iters[3]) > 20


@pytest.mark.parametrize("pf,db,form,rows", [(8, 1, 0, 0), (2, 2, 0, 0), (8, 2, 0, 0),
                                             (3, 1, 0, 0), (4, 1, 0, 0), (2, 1, 4, 64),
                                             (4, 1, 4, 32), (4, 1, 2, 64), (2, 1, 2, 32)])
def test_loop_kernel_variants_match_oracle(cuda, c0_oracle, pf, db, form, rows):
    # The CG loop's tunable kernel variants (the LLP kernel's loads through
    # the shared-memory ring, pf = 8, or 3 or 4 rows ahead in registers; the
    # lean two- and four-column walks, form = 2, 4, long and short; the
    # register-run blur-decimate, db = 2), forced through the recorded tuning:
    # the same Z0 and Z as the oracle, at the plain-form bar.
    sc, ref = c0_oracle
    cfg = sc["config"]
    hp = api.default_hrms_params(tol=1e-8, max_iter=5000)
    try:
        api.set_tuning(cfg.bands, cfg.H, cfg.W, cfg.ratio, 1, llp_pf=pf, db_impl=db,
                       llp_form=form, llp_rows=rows)
        Z, Z0, info = api.solve_hrms(to_dev(sc["lrms"], cuda), to_dev(sc["pan"], cuda),
                                     to_dev(sc["kernel"], cuda), cfg.ratio, hp, want_z0=True)
    finally:
        api.set_tuning(cfg.bands, cfg.H, cfg.W, cfg.ratio, 1)
    Z, Z0 = to_np(Z), to_np(Z0)
    assert all(s == 0 for s in info.status), info
    for b in range(cfg.bands):
        assert rel(Z0[b], ref["Z0"][b]) < PLAIN_TOL, b
        assert rel(Z[b], ref["Z"][b]) < PLAIN_TOL, b
