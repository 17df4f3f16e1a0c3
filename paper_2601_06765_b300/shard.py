"""Work distribution over ranks for the batched and served workloads.

The units of those workloads (independent systems, or one system modulo different primes) need no
data exchange: each rank runs its own share through its own context on its own GPU.  The only
cross-rank step is the reduction of what a benchmark reports (the slowest rank's time, the summed
counts).  Every rank computes the same partition from the same weights, so no communication decides
who runs what.
"""
from __future__ import annotations


def shard(weights: list[float], rank: int, world: int) -> list[int]:
    """Indices of the units rank `rank` of `world` runs, by greedy longest-processing-time
    assignment: units in order of decreasing weight (ties by index) go to the least-loaded rank
    (ties to the lower rank).  The shares partition range(len(weights)); each is ascending."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    load = [0.0] * world
    mine = []
    for i in sorted(range(len(weights)), key=lambda i: (-weights[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += weights[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def system_weight(system: dict) -> float:
    """Estimated cost of one system: the arena high-water fit the server's admission uses,
    2^(1.7 (d - 1) n) for n variables and input degree d (relative units)."""
    import numpy as np
    n = int(system["n"])
    d = int(np.asarray(system["exps"]).reshape(-1, n).sum(axis=1).max()) if len(system["exps"]) else 1
    return float(2.0 ** (1.7 * (max(d, 2) - 1) * n))


def aggregate(ms: float, count: float) -> tuple[float, float]:
    """(max over ranks of `ms`, sum over ranks of `count`) over the default process group, whatever
    its backend (NCCL between GPUs, gloo on CPU); (ms, count) when none is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(count)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    c = torch.tensor([float(count)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())
