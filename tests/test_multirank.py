"""Multi-rank host logic on CPU (gloo, world size 2): views are independent,
so ranks split a trajectory with no data-path collective; only the timing
maximum crosses ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2605_18334_gb300 import scenes
from paper_2605_18334_gb300.rasterizer import shard_views


def test_shard_views_partitions_and_balances():
    cams = scenes.trajectory_cameras(64)
    parts = [shard_views(cams, r, 4) for r in range(4)]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(64))
    load = [sum(cams[i]["width"] * cams[i]["height"] for i in p) for p in parts]
    assert max(load) - min(load) <= 1920 * 1080
    assert shard_views(cams, 0, 1) == list(range(64))
    with pytest.raises(ValueError):
        shard_views(cams, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    cams = scenes.trajectory_cameras(12)
    mine = shard_views(cams, rank, world)
    # each rank "times" its share; the job time is the slowest rank's
    t = float(sum(cams[i]["width"] * cams[i]["height"] for i in mine)) / 1e6
    tmax = bench.max_over_ranks(t, world)
    bench.barrier(world)
    q.put((rank, mine, t, tmax))
    dist.destroy_process_group()


def test_two_ranks_shard_views_and_reduce_timing_with_gloo():
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
    (r0, m0, t0, x0), (r1, m1, t1, x1) = res
    assert sorted(m0 + m1) == list(range(12)) and not set(m0) & set(m1)
    assert x0 == x1 == max(t0, t1)
