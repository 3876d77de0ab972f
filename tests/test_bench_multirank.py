"""Multi-rank aggregation of bench.py on CPU: two gloo ranks with different
frame times agree on the slowest one and report the whole job's throughput
(replicas, weak scaling, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, ms = bench.aggregate_ranks(2.0 + rank, 1920 * 1080, dist, "cpu")
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, ms in res:
        assert ms == 3.0                              # max over ranks
        assert abs(value - 2 * 1920 * 1080 / 3e-3 / 1e6) < 1e-6


def test_single_process_is_plain():
    import bench
    value, ms = bench.aggregate_ranks(1.5, 1000, None)
    assert ms == 1.5 and abs(value - 1000 / 1.5e-3 / 1e6) < 1e-12
