"""Host logic of the multi-GPU replicas path (no GPU): the longest-processing-time partition
of independent theta points and the gather of their results, run as world_size-2 gloo
process groups on the CPU with a stand-in evaluator."""
import os
import socket

import numpy as np
import pytest

from paper_2311_08050_gb300 import replicas


def test_partition_covers_every_unit_once_and_balances():
    rng = np.random.default_rng(7)
    sizes = rng.choice([512, 1024, 2048, 4096], size=64)
    costs = replicas.unit_costs(sizes, np.arange(64), 64)
    for world in (1, 2, 3, 4, 8):
        parts = replicas.partition_lpt(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [costs[p].sum() for p in parts]
        # LPT bound: max load <= 4/3 OPT, and OPT >= max(total / world, largest unit)
        opt_lb = max(costs.sum() / world, costs.max())
        assert max(loads) <= 4.0 / 3.0 * opt_lb + 1e-9


def test_partition_of_equal_units_is_round_robin_even():
    parts = replicas.partition_lpt([1.0] * 9, 2)
    assert sorted(len(p) for p in parts) == [4, 5]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_eval(idx):
    # stand-in for the GPU evaluation: a deterministic function of the unit index
    idx = np.asarray(idx)
    return -0.5 * idx.astype(np.float64) ** 2 + 3.0, (idx % 5 == 3).astype(np.int32) * -4


def _worker(rank, world, port, costs, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = replicas.evaluate_replicated(_fake_eval, costs, rank, world)
        t = replicas.max_over_ranks(1.0 + rank, world)
        q.put((rank, None if res is None else (res[0].tolist(), res[1].tolist()), t))
    finally:
        dist.destroy_process_group()


def test_gather_on_two_gloo_ranks_matches_single_process():
    import torch.multiprocessing as mp
    costs = [float(n) ** 3 for n in (4096, 512, 2048, 1024, 4096, 512, 512, 2048, 1024)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, res, t = q.get(timeout=120)
        out[rank] = (res, t)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref_lp, ref_st = _fake_eval(np.arange(len(costs)))
    lp, st = out[0][0]
    np.testing.assert_array_equal(np.asarray(lp), ref_lp)
    np.testing.assert_array_equal(np.asarray(st), ref_st)
    assert out[1][0] is None
    assert out[0][1] == out[1][1] == 2.0   # the slowest rank's time on every rank


def test_single_rank_needs_no_process_group():
    lp, st = replicas.evaluate_replicated(_fake_eval, [1.0, 2.0, 3.0], 0, 1)
    np.testing.assert_array_equal(lp, _fake_eval(np.arange(3))[0])
    assert replicas.max_over_ranks(2.5, 1) == 2.5
