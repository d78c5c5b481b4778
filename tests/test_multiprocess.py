"""The bench's multi-rank path on CPU: world_size 2 over gloo (127.0.0.1).

Each rank runs its own replica (replicas only: no collective on the data
path); the job's time is the slowest rank's, and the whole-job rate counts
the points of every rank.  Rank 0 alone prints the reference arm's line.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r's replica took (r + 1) seconds: the job took 2 s
        t = bench.max_over_ranks(float(rank + 1), world)
        rate = bench.whole_job_rate(1e9, 3, world, t)
        q.put((rank, t, rate, bench.dist_env()[:2]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_points():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]
    # 2 ranks x 3 steps x 1e9 points over 2 s = 3 GPts/s
    assert [o[2] for o in out] == [3.0, 3.0]
    assert [o[3] for o in out] == [(0, 2), (1, 2)]


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
