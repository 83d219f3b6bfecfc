"""bench.py's replica mode on CPU: two gloo ranks, each with its own timing;
the reported time is the slowest rank's and the throughput counts both
ranks' points."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.replica_throughput(10.0 + 5.0 * rank, 2_000_000_000, 4, world)
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 15.0
        assert value == pytest.approx(2e9 * 4 * 2 / 0.015 / 1e9)


def test_single_rank_is_local_time():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replica_throughput(8.0, 1_000_000, 10, 1)
    assert ms == 8.0 and value == pytest.approx(1e6 * 10 / 0.008 / 1e9)
