"""One system's force step shared out among several GPUs (group ranges).

The paper points to splitting the work over several GPUs for systems larger
than one GPU's memory or for more speed (§5).  The split built here keeps
the tree whole on every rank and shares out its groups:

* every rank holds the whole state (positions, velocities, masses) and
  builds the same tree (``bh_step_begin``: the build is deterministic, so the
  trees and the groups' order are identical);
* the groups are cut into one contiguous range per rank, balanced by an
  estimate of each group's walk cost (:func:`split_groups`): after a first
  step the previous step's interaction counts, spread over the bodies in
  sorted order (consecutive builds order the bodies almost alike), else the
  group sizes;
* each rank walks its own range (``bh_walk_groups``), then one collective
  per step gathers the accelerations of every rank's bodies into every
  rank's sorted force array (:func:`exchange`: an all-gather of each rank's
  contiguous body range, padded to the longest), and a second, small one
  the interaction counts of every rank's groups for the next split;
* every rank corrects every body (``bh_step_end``), so all ranks hold the
  same state again.

A walked group's forces do not depend on which rank walks it, so the step
equals the one-GPU step bit for bit.  The collectives are
``torch.distributed``'s (NCCL between GPUs, gloo on the host); the device
buffers are the context's own, never another GPU's memory.
"""
from __future__ import annotations

import numpy as np


def split_groups(cost, nranks: int):
    """Contiguous group ranges ``[(g0, g1), ...]``, one per rank, covering
    ``range(len(cost))`` in order and balancing the summed cost: rank r's
    range ends after the first group whose cumulative cost reaches (r + 1)/R
    of the total.  Every rank computes the same split from the same costs."""
    cost = np.asarray(cost, dtype=np.float64)
    G = len(cost)
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    cum = np.cumsum(cost)
    total = cum[-1] if G else 0.0
    bounds = [0]
    for r in range(1, nranks):
        b = int(np.searchsorted(cum, total * r / nranks, side="left")) + 1 if total > 0 else (G * r) // nranks
        bounds.append(min(max(b, bounds[-1]), G))
    bounds.append(G)
    return [(bounds[r], bounds[r + 1]) for r in range(nranks)]


def body_costs(gbeg, n_pc, n_pp):
    """Per-body walk cost of a finished walk, in sorted body order: each body
    of group g carries (n_pp + 2 n_pc) of its group's lists (a particle-cell
    interaction costs about twice a particle-particle one)."""
    gbeg = np.asarray(gbeg, dtype=np.int64)
    sizes = np.diff(gbeg)
    per = np.asarray(n_pp, dtype=np.float64) + 2.0 * np.asarray(n_pc, dtype=np.float64)
    return np.repeat(per, sizes)


def group_costs(gbeg, prev_body_cost=None):
    """Estimated walk cost of each group of the current build: the previous
    step's per-body costs summed over the group's sorted body range (clipped
    to the bodies that exist), else the group sizes."""
    gbeg = np.asarray(gbeg, dtype=np.int64)
    if prev_body_cost is None or len(prev_body_cost) == 0:
        return np.diff(gbeg).astype(np.float64)
    cum = np.concatenate([[0.0], np.cumsum(np.asarray(prev_body_cost, dtype=np.float64))])
    lo = np.minimum(gbeg[:-1], len(cum) - 1)
    hi = np.minimum(gbeg[1:], len(cum) - 1)
    return np.maximum(cum[hi] - cum[lo], 1.0)


def exchange(rows, ranges, rank: int, group=None):
    """All-gather of contiguous row ranges: ``rows`` is every rank's array of
    the same shape (a torch tensor, on the device for NCCL, on the host for
    gloo) whose rows ``ranges[rank]`` this rank computed; afterwards every
    rank's rows hold every rank's part.  Each part is padded to the longest
    range (an all-gather needs equal sizes)."""
    import torch
    import torch.distributed as dist

    world = len(ranges)
    longest = max((b - a for a, b in ranges), default=0)
    if world == 1 or longest == 0:
        return rows
    a, b = ranges[rank]
    mine = torch.zeros((longest,) + tuple(rows.shape[1:]), dtype=rows.dtype, device=rows.device)
    mine[: b - a] = rows[a:b]
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    for r, (a, b) in enumerate(ranges):
        if r != rank:
            rows[a:b] = parts[r][: b - a]
    return rows


class ShardedStep:
    """The leapfrog step of one system with its groups shared out among the
    ranks of ``torch.distributed``'s default group (or ``group``)."""

    def __init__(self, tc, rank: int, world: int, group=None):
        self.tc, self.rank, self.world, self.group = tc, rank, world, group
        self.prev_body_cost = None
        self.started = False
        self.last_ranges = None

    def _part(self, dt, theta, eps, init):
        import torch

        tc = self.tc
        tc.step_begin(dt, init=init)
        gbeg = tc.group_begins()
        ranges = split_groups(group_costs(gbeg, self.prev_body_cost), self.world)
        g0, g1 = ranges[self.rank]
        tc.walk_groups(theta, eps, g0, g1)
        body_ranges = [(int(gbeg[a]), int(gbeg[b])) for a, b in ranges]
        exchange(tc.sorted_forces(), body_ranges, self.rank, self.group)
        # the interaction counts of every rank's groups, for the next split
        st = tc.group_stats()
        counts = torch.from_numpy(np.stack([st["np"], st["nc"]], axis=1).astype(np.int64))
        if self.world > 1:
            dev = tc.sorted_forces().device if _backend_is_nccl(self.group) else torch.device("cpu")
            counts = exchange(counts.to(dev), ranges, self.rank, self.group).cpu()
        self.prev_body_cost = body_costs(gbeg, counts[:, 1].numpy(), counts[:, 0].numpy())
        tc.step_end(dt, init=init)
        self.last_ranges = ranges

    def step(self, dt: float, theta: float, eps: float):
        if not self.started:  # the accelerations at the loaded state first
            self._part(0.0, theta, eps, True)
            self.started = True
        self._part(dt, theta, eps, False)


def _backend_is_nccl(group=None) -> bool:
    import torch.distributed as dist

    return dist.is_initialized() and dist.get_backend(group) == "nccl"
