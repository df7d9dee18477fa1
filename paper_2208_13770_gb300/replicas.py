"""Runs over several GPUs of one node: one process per GPU.

The broad phase of one scene does not shard (the paper's method has no
exchange step), but a batch of independent scenes does: the scenes are
split over the ranks, greedily by particle count (shard_greedy), and every
rank advances its share with no collective on the data path.  The only
collectives are the timing ones: a barrier before the timed region and the
maximum of the ranks' times after it, so that the job's time is its
slowest rank's and its throughput counts the particle-steps of all ranks.
"""
from __future__ import annotations

import os


def rank_info(env=None):
    """(rank, world size, local rank) from the launcher's environment."""
    env = os.environ if env is None else env
    return (int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")),
            int(env.get("LOCAL_RANK", "0")))


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s replica: every rank runs its own scene."""
    return base + rank


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of `values` (floats) over all ranks of the default
    process group (identity on one rank)."""
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_throughput(world: int, n: int, steps: int, ms: float) -> float:
    """Units per second of the whole job: world ranks x n units x steps, over
    the slowest rank's time in milliseconds."""
    return world * n * steps / (ms * 1e-3)


def shard_greedy(sizes, world: int):
    """Scene indices of each rank: scenes taken largest first, each to the
    rank with the fewest particles so far (ties: the lowest rank); every
    rank's list in ascending scene order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    out = [[] for _ in range(world)]
    for q in sorted(range(len(sizes)), key=lambda q: (-int(sizes[q]), q)):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(q)
        load[r] += int(sizes[q])
    return [sorted(x) for x in out]
