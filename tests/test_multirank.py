"""The benchmark's multi-rank path (replicas only) on CPU ranks with gloo:
time is the maximum over ranks and points the sum, as rank 0 reports them."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, pts = bench.aggregate(1.0 + rank, 100.0 * (rank + 1), world)
    bench.barrier(world)
    q.put((rank, ms, pts))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
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
    for rank, ms, pts in res:
        assert ms == 2.0      # max over ranks
        assert pts == 300.0   # sum over ranks


def test_single_rank_aggregate_is_identity():
    import bench
    assert bench.aggregate(3.5, 7.0, 1) == (3.5, 7.0)
