"""The multi-process path of bench.py (replicas: one process per GPU, max of
the per-rank times, sum of the work) exercised on CPU with gloo, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp
from mp_util import collect


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    t = bench.max_over_ranks(dist, 1.5 + rank)  # per-rank "time"
    q.put((rank, t))
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(collect(q, procs, 2, 300))
    assert out == {0: 2.5, 1: 2.5}


def test_replica_value_is_sum_of_work_over_max_time():
    import bench

    b = bench.site_bytes("f32-full", 1)
    assert b == 40 * 72 + 192
    assert bench.site_bytes("f64-full", 1) == 6144
    assert bench.site_bytes("f16-2row", 12) == 960 + 12 * 192
