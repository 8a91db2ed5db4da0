"""The benchmark's multi-rank aggregation with world_size 2 over gloo (CPU).

Each rank runs an independent beam replica; the whole-job rate is all ranks'
units over the slowest rank's time. No GPU is needed here.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = [2.0, 3.0][rank]
    slowest = bench.max_over_ranks(local_seconds, "cpu")
    rate = bench.aggregate_throughput(1000, 10, world, slowest)
    dist.barrier()
    q.put((rank, slowest, rate))
    dist.destroy_process_group()


def test_two_rank_aggregation_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == 3.0
        assert rate == pytest.approx(2 * 1000 * 10 / 3.0)


def test_single_process_aggregation():
    import bench
    assert bench.max_over_ranks(1.5, "cpu") == 1.5
    assert bench.aggregate_throughput(4096 * 65536, 200, 1, 2.0) == pytest.approx(4096 * 65536 * 100)
