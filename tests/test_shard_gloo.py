"""The multi-rank path of the batched and served workloads, on CPU: the share of each rank
(paper_2601_06765_b300.shard.shard) and the reduction of the reported numbers across ranks
(shard.aggregate) with two gloo ranks.  No GPU: the data path has no collective, so the host logic
is all there is to test across processes."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

from paper_2601_06765_b300 import shard, synth


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shares_partition_and_balance(world):
    rng = np.random.default_rng(world)
    weights = list(rng.pareto(1.5, size=200) + 1.0)
    shares = [shard.shard(weights, r, world) for r in range(world)]
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(len(weights)))
    # greedy longest-first: no rank exceeds the average by more than the largest unit
    loads = [sum(weights[i] for i in s) for s in shares]
    assert max(loads) <= sum(weights) / world + max(weights) + 1e-9
    assert all(s == sorted(s) for s in shares)


def test_equal_units_split_evenly_and_deterministically():
    w = [1.0] * 128  # the 128-prime batch: one system modulo 128 primes
    a = [shard.shard(w, r, 2) for r in range(2)]
    assert [len(x) for x in a] == [64, 64]
    assert a == [shard.shard(w, r, 2) for r in range(2)]


def test_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.shard([1.0], 2, 2)


def test_system_weight_orders_by_size():
    small = synth.dense_system(5, 5, 65521, 1)
    big = synth.dense_system(9, 9, 65521, 1)
    cubic = synth.dense_system(5, 5, 65521, 1, degree=3)
    assert shard.system_weight(small) < shard.system_weight(big)
    assert shard.system_weight(small) < shard.system_weight(cubic)


def _worker(rank: int, world: int, port: int, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        systems = synth.mixed_batch(24)
        weights = [shard.system_weight(s) for s in systems]
        mine = shard.shard(weights, rank, world)
        # each rank "runs" its share: a time that differs per rank and a count per unit
        ms, count = shard.aggregate(10.0 * (rank + 1), float(len(mine)))
        q.put((rank, mine, ms, count))
    finally:
        dist.destroy_process_group()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_share_and_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    shares = [g[1] for g in got]
    assert sorted(shares[0] + shares[1]) == list(range(24))
    assert not set(shares[0]) & set(shares[1])
    for _, _, ms, count in got:
        assert ms == 20.0          # the slower rank's time
        assert count == 24.0       # all ranks' units
    # without a process group the numbers pass through unchanged
    assert shard.aggregate(3.0, 5.0) == (3.0, 5.0)
