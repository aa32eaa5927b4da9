"""Evaluation of the learned warm start on held-out scenes, on the GPU with
the library's own kernels.

Protocol: seeded synthetic 8-band, ratio-4 scenes from the training
generator (anisotropic 17 x 17 kernels; shape density of the 1024^2
workload, i.e. the shape count scaled with the area), never seen in training
(seeds 5000 and up; training uses 1000-2999). For every scene the kernel is
estimated (Algorithm 1), then Z0 (Eq. Z_ini_matting) is solved to the same
relative residual from zeros (the cold start) and from the network's output
(the warm start), with the FFT alias-group preconditioned CG and with plain
CG, and the Z step follows (Eq. Z_solution). Reported per scene and in
aggregate: CG iterations per band, the per-band rel-L2 of the warm-start
HRMS against the cold-start HRMS and of both against a solve to 1e-9, and
the device time of the two solves. Usage:

    python -m paper_2103_09943_gb300.eval_warm --weights weights/warm_cnn.npz --out eval.json
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import replace

import numpy as np
import torch

from . import api
from .cnn import WarmStartNet


def scene_configs(count: int, size: int, seed0: int):
    import synth
    base = synth.CONFIGS["c1"]
    shapes = max(8, int(round(base.shapes * (size * size) / (base.H * base.W))))
    return [replace(base, name=f"heldout_{seed0 + k}", H=size, W=size, shapes=shapes,
                    seed=seed0 + k) for k in range(count)]


def _rel(a: torch.Tensor, b: torch.Tensor) -> list:
    d = (a.double() - b.double()).flatten(1).norm(dim=1)
    return (d / b.double().flatten(1).norm(dim=1)).tolist()


def evaluate_scene(X, Y, cfg, net, tol: float, dev):
    """Cold and warm solves of one scene; per-band iterations, errors, times."""
    ratio, R = cfg.ratio, cfg.R
    kern, _, kinfo = api.estimate_kernel(X, Y, ratio, R)
    out = {"seed": cfg.seed, "admm_iters": kinfo.iters}
    p_ref = api.default_hrms_params(tol=1e-9, max_iter=20000)
    z_ref, _, _ = api.solve_hrms(X, Y, kern, ratio, p_ref)
    for name, precond in (("pcg", 1), ("plain_cg", 0)):
        res = {}
        for start, warm in (("cold", 0), ("warm", 2)):
            hp = api.default_hrms_params(tol=tol, precond=precond, warm=warm, max_iter=20000,
                                         cnn_params=net.params.data_ptr() if warm else None)
            ws = api.workspace(cfg.bands, cfg.H, cfg.W, ratio, R, dev, hp)
            api.solve_hrms(X, Y, kern, ratio, hp, ws=ws, info=False)     # graphs built
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            z, _, info = api.solve_hrms(X, Y, kern, ratio, hp, ws=ws)
            b.record()
            torch.cuda.synchronize()
            res[start] = {"iters": info.iters, "ms": a.elapsed_time(b), "z": z,
                          "status": info.status}
        out[name] = {
            "iters_cold": res["cold"]["iters"], "iters_warm": res["warm"]["iters"],
            "ms_cold": res["cold"]["ms"], "ms_warm": res["warm"]["ms"],
            "rel_l2_warm_vs_cold": _rel(res["warm"]["z"], res["cold"]["z"]),
            "rel_l2_cold_vs_tight": _rel(res["cold"]["z"], z_ref),
            "rel_l2_warm_vs_tight": _rel(res["warm"]["z"], z_ref),
            "status_ok": all(s == 0 for s in res["cold"]["status"] + res["warm"]["status"]),
        }
    return out


def summarize(rows: list) -> dict:
    summ = {}
    for name in ("pcg", "plain_cg"):
        ic = np.array([i for r in rows for i in r[name]["iters_cold"]], dtype=float)
        iw = np.array([i for r in rows for i in r[name]["iters_warm"]], dtype=float)
        msc = np.array([r[name]["ms_cold"] for r in rows])
        msw = np.array([r[name]["ms_warm"] for r in rows])
        summ[name] = {
            "bands": int(ic.size),
            "iters_cold_mean": float(ic.mean()), "iters_warm_mean": float(iw.mean()),
            "iters_saved_pct": float(100.0 * (1.0 - iw.sum() / ic.sum())),
            "iters_warm_p90": float(np.percentile(iw, 90)),
            "solve_ms_cold_mean": float(msc.mean()), "solve_ms_warm_mean": float(msw.mean()),
            "time_saved_pct": float(100.0 * (1.0 - msw.sum() / msc.sum())),
            "rel_l2_warm_vs_cold_max": float(max(max(r[name]["rel_l2_warm_vs_cold"])
                                                 for r in rows)),
            "rel_l2_cold_vs_tight_max": float(max(max(r[name]["rel_l2_cold_vs_tight"])
                                                  for r in rows)),
            "rel_l2_warm_vs_tight_max": float(max(max(r[name]["rel_l2_warm_vs_tight"])
                                                  for r in rows)),
            "all_converged": all(r[name]["status_ok"] for r in rows),
        }
    return summ


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--weights", required=True)
    ap.add_argument("--scenes", type=int, default=64)
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--seed0", type=int, default=5000)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--out", default=None, help="JSON file for the per-scene results")
    args = ap.parse_args(argv)
    import synth
    cfgs = scene_configs(args.scenes, args.size, args.seed0)
    t0 = time.time()
    arrays = synth.make_scenes_parallel(cfgs)       # host cores, before any CUDA call
    t_gen = time.time() - t0
    dev = torch.device("cuda")
    net = WarmStartNet.load(args.weights, device=dev)
    rows = []
    t0 = time.time()
    for cfg, (lrms, pan) in zip(cfgs, arrays):
        X = torch.from_numpy(lrms).to(dev)
        Y = torch.from_numpy(pan).to(dev)
        rows.append(evaluate_scene(X, Y, cfg, net, args.tol, dev))
    rec = {"protocol": f"{args.scenes} held-out scenes, seeds {args.seed0}-"
                       f"{args.seed0 + args.scenes - 1}, 8 x {args.size}^2, ratio 4, "
                       f"17 x 17 kernels estimated; Z0 to relative residual {args.tol}",
           "weights": args.weights, "host_generation_s": t_gen,
           "gpu_s": time.time() - t0, "summary": summarize(rows)}
    print(json.dumps(rec, indent=1), flush=True)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump({**rec, "scenes": rows}, fh)


if __name__ == "__main__":
    main()
