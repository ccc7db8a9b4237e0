"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2):
every rank gets its own replica of the inputs, timing is reduced with a MAX
over ranks, and the whole-job rate counts the units of all ranks.  No GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 1.0 + 2.0 * rank                      # rank 1 is the slow one
        worst = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        wl = bench.WORKLOADS["1d4096"]
        x = bench.make_input(wl, bench.replica_rep(rank, 0))
        digest = float(np.abs(x[:4]).sum())
        out = [None] * world
        dist.all_gather_object(out, digest)
        rate = bench.whole_job_rate(world, 100.0, worst)
        q.put((rank, worst, out, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, worst, digests, rate in res:
        assert worst == 3.0                        # max over ranks, seen by every rank
        assert digests[0] != digests[1]            # each rank transforms different data
        assert rate == pytest.approx(2 * 100.0 / 3.0e-3)


def test_single_process_helpers():
    assert bench.max_over_ranks(2.5, None, None) == 2.5
    assert bench.whole_job_rate(1, 10.0, 1000.0) == pytest.approx(10.0)
    assert len({bench.replica_rep(r, b) for r in range(8) for b in range(8)}) == 64


def _run_bench(env_extra):
    import json
    import subprocess
    import sys
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"), "--impl",
                        "reference", "--steps", "1", "--warmup", "3", "--workload", "1d4096"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    return [json.loads(l) for l in lines]


def test_reference_arm_prints_one_line_on_rank0_only():
    out0 = _run_bench({"RANK": "0", "WORLD_SIZE": "2"})
    assert len(out0) == 1 and out0[0]["impl"] == "reference"
    line = out0[0]
    assert line["unit"] == "GB/s" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["n_gpus"] == 2
    assert _run_bench({"RANK": "1", "WORLD_SIZE": "2"}) == []
