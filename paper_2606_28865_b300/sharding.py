"""Partitioning the long-range evaluation across ranks (one process per GPU, torch.distributed).

The evaluation shards at two levels:

* Independent evaluations (the instances of a batch, serving requests, the alphas of a Rothe
  step) shard by instance with no data exchange: ``assign_instances`` balances their costs
  (longest processing time first), every rank evaluates its own share and
  ``evaluate_instances`` gathers the results on every rank.
* One evaluation shards by source.  The type-1 step (Section 5.2, eq. disrete_sigma_hat) is linear
  in the strengths, so each rank forms the spread quantity of its own source shard (the grid, or
  any linear function of it such as its transform), a single all-reduce (sum) of that quantity is
  the method's only exchange step, and each rank then finishes the evaluation (multiplier,
  inverse transform, type-2 step) at its own target shard.  ``evaluate_source_sharded`` runs that
  scheme.

The compute is passed in as callables, so the same partitioning serves ranks on GPUs (the
library's kernels, NCCL) and ranks on CPU cores (gloo).  ``pg`` is the ``torch.distributed``
module (initialised) or None for a single process.
"""
from __future__ import annotations

import heapq

import numpy as np


def _rank_world(pg):
    if pg is None:
        return 0, 1
    return pg.get_rank(), pg.get_world_size()


def split_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous share [lo, hi) of n items for one rank (shares differ by at most one)."""
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def assign_instances(costs, world: int) -> list[list[int]]:
    """Instances per rank: longest processing time first, each to the least loaded rank (ties to
    the lower rank), so the assignment is the same on every rank."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(x) for x in out]


def evaluate_instances(costs, eval_fn, pg=None) -> dict:
    """Evaluate instance i by eval_fn(i) on the rank it is assigned to; every rank returns
    {i: result} for all instances (results are gathered as Python objects)."""
    rank, world = _rank_world(pg)
    mine = {i: eval_fn(i) for i in assign_instances(costs, world)[rank]}
    if pg is None:
        return mine
    parts = [None] * world
    pg.all_gather_object(parts, mine)
    out = {}
    for p in parts:
        out.update(p)
    return out


def evaluate_source_sharded(n_src: int, n_trg: int, partial_fn, finish_fn, pg=None) -> np.ndarray:
    """One evaluation sharded by source and by target.

    partial_fn(lo, hi) -> tensor: the spread quantity of sources [lo, hi) (a torch tensor on the
        device the process group reduces on);
    finish_fn(total, lo, hi) -> array: the potential at targets [lo, hi) from the summed quantity.
    Returns the potential at all n_trg targets on every rank."""
    rank, world = _rank_world(pg)
    lo, hi = split_range(n_src, world, rank)
    part = partial_fn(lo, hi)
    if pg is not None:
        pg.all_reduce(part)  # sum over the source shards: the one exchange step
    tlo, thi = split_range(n_trg, world, rank)
    u = np.asarray(finish_fn(part, tlo, thi), dtype=np.float64)
    if pg is None:
        return u
    parts = [None] * world
    pg.all_gather_object(parts, u)
    return np.concatenate(parts)
