"""The N > 1 benchmark path runs independent replicas: no data exchange, and the job's
time is the slowest rank's.  Checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 if rank == 0 else 250.0          # rank 1 is the slow one
    q.put((rank, bench.job_throughput(ms, 1_000_000)))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms_max, value = got[r]
        assert ms_max == 250.0
        assert value == pytest.approx(2 * 1_000_000 / 0.25 / 1e6)


def test_one_process_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, value = bench.job_throughput(50.0, 500_000)
    assert ms_max == 50.0 and value == pytest.approx(10.0)
