"""The bench's multi-rank arithmetic, on two gloo ranks on the CPU: the timed
region is the slowest rank's, replica rates add up, the whole-job rate counts
every rank's events; and the reference arm does no work on ranks other than 0."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench

    ms = bench.max_over_ranks(dist, torch, 10.0 + 3.0 * rank, "cpu")
    vals = bench.sum_over_ranks(dist, torch, [1e9 * (rank + 1), 0.5], "cpu")
    rate = bench.whole_job_rate(4, 1 << 20, world, ms)
    q.put((rank, ms, vals, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(g[0] for g in got) == [0, 1]
    for _, ms, vals, rate in got:
        assert ms == 13.0  # the slower rank's time, on every rank
        assert vals == [3e9, 1.0]
        assert rate == pytest.approx(4 * (1 << 20) * 2 / 0.013)


def test_reference_arm_is_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
