"""Multi-GPU evaluation by replicas: one process per GPU, no data-path collective.

Every theta point (or model) is an independent unit of work -- the Laplace evaluation of
one hyperparameter configuration -- so the units are partitioned across ranks and each rank
runs its share through its own GPU.  The only exchange is a gather of the per-unit results
(log pi~(theta|y), status, optionally the mode and the variances) at the end.  The partition
is longest-processing-time-first on the unit costs (n^3 of the unit's model: the dense
factorisations dominate), which keeps the slowest rank within 4/3 of the optimum.

The evaluator is a callable so that the host logic runs (and is tested) without a GPU.
"""
from __future__ import annotations

import heapq
from typing import Callable, Sequence

import numpy as np


def partition_lpt(costs: Sequence[float], world: int) -> list[list[int]]:
    """Assign unit indices to `world` ranks, largest cost first to the least-loaded rank.
    Ties go to the lowest rank; every rank's list is returned in increasing index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def unit_costs(model_sizes: Sequence[int], model_of_theta: Sequence[int] | None, nunits: int) -> np.ndarray:
    """Cost of each theta point: n^3 of its model."""
    n = np.asarray(model_sizes, dtype=np.float64)
    idx = np.zeros(nunits, dtype=np.int64) if model_of_theta is None else np.asarray(model_of_theta, dtype=np.int64)
    return n[idx] ** 3


def evaluate_replicated(evaluate: Callable[[np.ndarray], tuple[np.ndarray, np.ndarray]], costs: Sequence[float],
                        rank: int, world: int, group=None) -> tuple[np.ndarray, np.ndarray] | None:
    """Evaluate this rank's share of the units and gather every result on rank 0.

    `evaluate(indices)` returns (log_post, status) for the given unit indices (in that order).
    Rank 0 receives the full arrays in the original unit order; the other ranks receive None.
    With world == 1 no process group is needed."""
    parts = partition_lpt(costs, world)
    mine = np.asarray(parts[rank], dtype=np.int64)
    lp, st = evaluate(mine) if len(mine) else (np.zeros(0), np.zeros(0, dtype=np.int32))
    lp = np.asarray(lp, dtype=np.float64)
    st = np.asarray(st, dtype=np.int32)
    if world == 1:
        return lp, st
    import torch
    import torch.distributed as dist
    # fixed-size exchange: every rank sends (index, log_post, status) rows padded to the
    # largest share, so a plain all_gather of one tensor suffices
    width = max(len(p) for p in parts)
    buf = torch.full((width, 3), float("nan"), dtype=torch.float64)
    if len(mine):
        buf[: len(mine), 0] = torch.from_numpy(mine.astype(np.float64))
        buf[: len(mine), 1] = torch.from_numpy(lp)
        buf[: len(mine), 2] = torch.from_numpy(st.astype(np.float64))
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    if rank != 0:
        return None
    n = len(costs)
    out_lp = np.full(n, np.nan)
    out_st = np.full(n, -1, dtype=np.int32)
    for b in bufs:
        rows = b.numpy()
        rows = rows[~np.isnan(rows[:, 0])]
        idx = rows[:, 0].astype(np.int64)
        out_lp[idx] = rows[:, 1]
        out_st[idx] = rows[:, 2].astype(np.int32)
    return out_lp, out_st


def max_over_ranks(t: float, world: int, group=None) -> float:
    """The slowest rank's time (the job's time): all-reduce MAX over the ranks."""
    if world == 1:
        return float(t)
    import torch
    import torch.distributed as dist
    x = torch.tensor([float(t)], dtype=torch.float64)
    dist.all_reduce(x, op=dist.ReduceOp.MAX, group=group)
    return float(x.item())
