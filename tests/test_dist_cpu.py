"""Multi-rank host logic on CPU with the gloo backend (world size 2): the
max-over-ranks timing and unit totals the benchmark reports, and the
deterministic split of an ensemble's runs across ranks."""
import os
import socket

import pytest

from paper_2312_05410_gb300.dist import aggregate, shard_runs

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sec, units = aggregate(1.0 + rank, 10.0 * (rank + 1))
        mine = shard_runs(costs, world, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, sec, units, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard():
    import torch.multiprocessing as mp

    costs = [128 * 128, 512 * 512, 256 * 256, 192 * 192, 384 * 384, 512 * 512, 128 * 128]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, sec, units, gathered in out:
        assert sec == 2.0 and units == 30.0  # max time, total units
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(len(costs)))  # every run on exactly one rank
        assert gathered == [shard_runs(costs, 2, r) for r in range(2)]  # same split on every rank


def test_shard_balance_and_single_rank():
    costs = [5, 3, 3, 2, 2, 1]
    assert shard_runs(costs, 1, 0) == list(range(6))
    parts = [shard_runs(costs, 2, r) for r in range(2)]
    loads = [sum(costs[i] for i in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(costs)
    with pytest.raises(ValueError):
        shard_runs(costs, 2, 2)


def test_aggregate_without_process_group_is_identity():
    assert aggregate(1.5, 7.0) == (1.5, 7.0)
