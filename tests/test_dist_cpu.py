"""Host logic of the multi-rank benchmark on CPU: world_size 2 gloo ranks.

Scenes are independent units, so the benchmark runs one replica per rank with
no collective on the data path; only the timing reduction (max over ranks)
and the barrier use torch.distributed. These checks need no GPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        # per-rank step times: the job time is the slowest rank
        t = bench.reduce_max(10.0 + rank, w, device="cpu")
        bench.barrier(w)
        # weak scaling: each rank processes its own scene
        cfg = bench.workload_config(1)
        units = cfg.bands * cfg.H * cfg.W
        value = bench.throughput(units, w, t * 1e-3)
        # each rank draws a different scene (seed + rank)
        import synth
        from dataclasses import replace
        small = replace(synth.CONFIGS["c0"], H=64, W=64, shapes=5, seed=100 + r)
        sc = synth.make_scene(small)
        q.put((r, w, t, value, float(sc["pan"].sum())))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction_and_weak_scaling():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    # max over ranks on every rank
    assert all(o[2] == 11.0 for o in out)
    # whole-job throughput counts both replicas
    import bench
    cfg = bench.workload_config(1)
    expect = 2 * cfg.bands * cfg.H * cfg.W / 1e6 / 11e-3
    assert all(abs(o[3] - expect) < 1e-6 * expect for o in out)
    # independent scenes per rank
    assert out[0][4] != out[1][4]


def test_single_rank_helpers_are_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)
    assert bench.throughput(1e6, 1, 1.0) == pytest.approx(1.0)
