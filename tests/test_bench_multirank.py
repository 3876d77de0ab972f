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


def _tile_worker(rank, world, port, q):
    """Rank r computes the stage 1-2 pairs of its band of rows of one frame
    through the window parameters (host execution of the device code); the
    bands are gathered on every rank."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import bench
    from paper_1404_3363_gb300 import ivv, scenes
    sc = scenes.config(2, width=96, height=60)
    y0, h = bench.tile_rows(sc.height, rank, world)
    cnt, pairs, blk = ivv.host_render_pairs(sc.blocks, sc.scalar_mode, sc.camera, sc.params, sc.width, h,
                                            max_pairs=4, window=(0, y0, sc.width, sc.height))
    mine = torch.from_numpy(np.concatenate([cnt.astype(np.float64), pairs.reshape(-1), blk.reshape(-1)]))
    sizes = [None] * world
    dist.all_gather_object(sizes, (y0, h, mine.numel()))
    bufs = _gather_uneven(mine, sizes)
    if rank == 0:
        q.put([(y0_, h_, b.numpy()) for (y0_, h_, _), b in zip(sizes, bufs)])
    dist.barrier()
    dist.destroy_process_group()


def _gather_uneven(t, sizes):
    n_max = max(n for _, _, n in sizes)
    padded = torch.zeros(n_max, dtype=torch.float64)
    padded[:t.numel()] = t
    out = [torch.zeros(n_max, dtype=torch.float64) for _ in sizes]
    dist.all_gather(out, padded)
    return [o[:n] for o, (_, _, n) in zip(out, sizes)]


def test_two_ranks_rendering_row_bands_tile_the_frame():
    """Screen tiles per GPU (the frame split that bench.py --split rows uses):
    two gloo ranks compute the entry/exit pairs of their row bands through
    the window parameters; assembled, they equal the one-call frame exactly."""
    import numpy as np
    from paper_1404_3363_gb300 import ivv, scenes
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_tile_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    sc = scenes.config(2, width=96, height=60)
    cnt, pairs, blk = ivv.host_render_pairs(sc.blocks, sc.scalar_mode, sc.camera, sc.params, sc.width, sc.height,
                                            max_pairs=4)
    W = sc.width
    rows_cnt = np.zeros(sc.height * W)
    rows_pairs = np.zeros((4, sc.height * W, 8))
    rows_blk = np.zeros((4, sc.height * W))
    covered = 0
    for y0, h, flat in got:
        n = h * W
        c = flat[:n]
        pr = flat[n:n + 4 * n * 8].reshape(4, n, 8)
        bk = flat[n + 4 * n * 8:].reshape(4, n)
        rows_cnt[y0 * W:(y0 + h) * W] = c
        rows_pairs[:, y0 * W:(y0 + h) * W] = pr
        rows_blk[:, y0 * W:(y0 + h) * W] = bk
        covered += h
    assert covered == sc.height
    assert (cnt > 0).sum() > 100
    np.testing.assert_array_equal(rows_cnt, cnt)
    np.testing.assert_array_equal(rows_pairs, pairs)
    np.testing.assert_array_equal(rows_blk, blk)
