"""The multi-GPU path of the benchmark is replicas only (independent domains
per rank, no data-path collective); its host logic -- the max-over-ranks
timing reduction, the whole-job throughput and the rank-0-only reference
arm -- runs here as world-size-2 gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank times its replica; the job is as slow as the slowest rank
    slowest = bench.max_over_ranks(dist, 10.0 + rank)
    dist.barrier()
    out.put((rank, slowest, bench.whole_job_mlups(1000, 5, world, slowest)))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the maximum; value = all ranks' cell updates / that time
    assert [r[1] for r in res] == [11.0, 11.0]
    expected = 1000 * 5 * 2 / 11e-3 / 1e6
    assert all(abs(r[2] - expected) < 1e-12 for r in res)


def test_whole_job_value_is_weak_scaling():
    import bench
    one = bench.whole_job_mlups(24_000_000, 200, 1, 250.0)
    two = bench.whole_job_mlups(24_000_000, 200, 2, 250.0)
    assert abs(two - 2 * one) < 1e-9


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
