"""The benchmark's multi-rank path on CPU (gloo, world size 2): every rank runs
its own system, and only the timing is combined -- the slowest rank's time and
the sum of the bodies of all ranks (weak scaling, no collective on the data
path)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env()[:2] == (rank, world)
        t = bench.max_over_ranks(10.0 + rank, world)  # ms of each rank
        b = bench.sum_over_ranks(1000.0 * (rank + 1), world)  # bodies of each rank
        out.put((rank, t, b))
    finally:
        dist.destroy_process_group()


def test_two_ranks_combine_timing():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 11.0, 3000.0), (1, 11.0, 3000.0)]
