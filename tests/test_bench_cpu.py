"""Host-side pieces of the benchmark: the launch count it claims for a step
(against a count written out by hand for one configuration) and the JSON
line of its reference arm, the FP64 oracle on the host cores."""
import importlib.util
import json
import os
import subprocess
import sys
from types import SimpleNamespace

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_launch_count_by_hand():
    b = _bench()
    cfg = synth.CONFIGS["c1"]                       # 8 bands, 17 x 17 kernel
    hp = SimpleNamespace(precond=1, zstep_fp32=1, warm=2)
    iters = [47, 50, 44, 47, 48, 44, 47, 47]
    # kernel estimate: omega 4, f + lags + assembly + E^T f 4, Cholesky of
    # 289 unknowns in 10 panels (add_diag, 10 diagonal tiles, 9 panels, 9
    # updates), solve, inverse, ADMM, status collector
    kest = 4 + 4 + (1 + 10 + 9 + 9) + 3 + 1
    # four branch loops of band pairs; maxima 50, 47, 48, 47 -> 13, 12, 12, 12
    # bodies of four iterations of 7 kernels
    loop = 7 * 4 * (13 + 12 + 12 + 12)
    # PAN stats, spectrum 4, rhs, reset, init, z0 = P^-1 r0 (3), FP32 Z step 4,
    # status collector
    solve = 1 + 4 + 1 + 2 + 3 + loop + 4 + 1
    warm = 1 + 9 + 2
    assert b.launches_per_step(cfg, hp, iters, 4) == kest + solve + warm
    # one loop over all bands: max 50 -> 13 bodies
    assert b.launches_per_step(cfg, hp, iters, 1) == kest + solve - loop + 7 * 4 * 13 + warm


def test_batch_launch_count():
    # one timer stamp, then per scene the one-scene count with all its bands
    # in one loop (split 1) and its own stamp
    b = _bench()
    cfgs = synth.make_batch_configs(3, 3000)
    hp = SimpleNamespace(precond=1, zstep_fp32=1, warm=2)
    sinfo = [SimpleNamespace(iters=[40 + k] * c.bands) for k, c in enumerate(cfgs)]
    want = 1 + sum(b.launches_per_step(c, hp, [40 + k] * c.bands, 1) + 1
                   for k, c in enumerate(cfgs))
    assert b.batch_launches(cfgs, hp, sinfo) == want


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--ref-crop", "32"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "Mpix·band/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]
    # the same config as the GPU arm's line (the workload, not a crop of it)
    b = _bench()
    args = b.parse(["--ref-crop", "32"])
    assert d["config"] == b.batch_config(synth.make_batch_configs(args.batch, 3000), args)
