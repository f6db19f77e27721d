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


# ------------------------------------------- one system, groups shared out
def _shard_rank(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1106_1900_gb300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the same build on every rank: 40 groups of uneven sizes over their sorted bodies
        rng = np.random.default_rng(7)
        sizes = rng.integers(1, 50, 40)
        gbeg = np.concatenate([[0], np.cumsum(sizes)])
        n = int(gbeg[-1])
        prev = rng.uniform(1.0, 5.0, n)  # the previous step's per-body costs
        ranges = shard.split_groups(shard.group_costs(gbeg, prev), world)
        # host stand-in for the sorted force array: this rank fills its own bodies only
        rows = torch.full((n, 4), -1.0)
        a, b = int(gbeg[ranges[rank][0]]), int(gbeg[ranges[rank][1]])
        rows[a:b] = torch.arange(a, b, dtype=torch.float32)[:, None] * torch.tensor([1.0, 2.0, 3.0, 4.0])
        body_ranges = [(int(gbeg[g0]), int(gbeg[g1])) for g0, g1 in ranges]
        shard.exchange(rows, body_ranges, rank)
        out.put((rank, ranges, rows.numpy().tolist()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_out_groups_and_gather_forces():
    """The split of one system's groups and the exchange of the walked bodies'
    forces (gloo, world size 2, host tensors standing in for the device
    arrays): both ranks compute the same contiguous split, and after the
    all-gather both hold every body's row."""
    import numpy as np
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q), daemon=True) for r in range(2)]
    for p in procs:
        p.start()
    # read the results before joining: a rank cannot exit while its result still fills the pipe
    got = sorted((q.get(timeout=120) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (r0, ranges0, rows0), (r1, ranges1, rows1) = got
    assert ranges0 == ranges1 and ranges0[0][0] == 0 and ranges0[0][1] == ranges0[1][0] and ranges0[1][1] == 40
    want = np.arange(len(rows0))[:, None] * np.array([1.0, 2.0, 3.0, 4.0])
    assert np.array_equal(np.array(rows0), want) and np.array_equal(np.array(rows1), want)


def test_split_balances_costs():
    import numpy as np

    from paper_1106_1900_gb300 import shard

    rng = np.random.default_rng(3)
    cost = rng.uniform(1.0, 10.0, 1000)
    for R in (1, 2, 3, 8):
        rs = shard.split_groups(cost, R)
        assert rs[0][0] == 0 and rs[-1][1] == 1000 and all(rs[i][1] == rs[i + 1][0] for i in range(R - 1))
        loads = [cost[a:b].sum() for a, b in rs]
        assert max(loads) - min(loads) <= 2 * cost.max()  # within a group or two of even
    # more ranks than groups: empty ranges, still a cover
    rs = shard.split_groups([1.0, 1.0], 4)
    assert rs[0][0] == 0 and rs[-1][1] == 2 and sum(b - a for a, b in rs) == 2
    # per-body costs from a walk, summed over the next build's groups
    gbeg = np.array([0, 3, 5, 9])
    bc = shard.body_costs(gbeg, n_pc=[1, 2, 3], n_pp=[10, 20, 30])
    assert bc.tolist() == [12.0] * 3 + [24.0] * 2 + [36.0] * 4
    assert shard.group_costs(np.array([0, 4, 9]), bc).tolist() == [12.0 * 3 + 24.0, 24.0 + 36.0 * 4]
    assert shard.group_costs(gbeg).tolist() == [3.0, 2.0, 4.0]
