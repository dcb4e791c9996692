"""Rank bookkeeping of the benchmark's N > 1 path, on CPU with gloo.

The single-mask path does not shard: N ranks run independent replicas and
the only cross-rank traffic is the barrier around the timed region and the
max over ranks of the step time.  These tests run that bookkeeping with two
gloo ranks (no GPU), and check that the reference arm's non-zero ranks exit
without work.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, step_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, loc = bench.dist_setup(backend="gloo")
    assert (w, r, loc) == (world, rank, rank)
    bench.barrier(w)
    ms = bench.max_over_ranks(step_ms[rank], w)
    out.put((rank, ms, bench.job_throughput(1000.0, ms, w)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world = 2
    step_ms = [1.5, 4.0]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, step_ms, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; throughput counts the units of all ranks
    assert [g[1] for g in got] == [4.0, 4.0]
    assert all(g[2] == pytest.approx(2 * 1000.0 / 4e-3) for g in got)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_throughput(10.0, 2.0, 1) == pytest.approx(5000.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
