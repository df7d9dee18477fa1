"""The multi-GPU path on CPU: world size 2 over gloo (127.0.0.1).

The batch's scenes are split over the ranks (greedily by particle count);
the job's time is the maximum over the ranks and its throughput counts
every rank's particle-steps.  Here each rank takes its share of the 512
scenes and reports a different time; both must see the same maxima, the
shares must cover every scene once, and the particle counts summed over
the ranks must be the batch's.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2208_13770_gb300 import replicas
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = replicas.rank_info()
        assert (r, w, loc) == (rank, world, rank)
        mx = replicas.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5])
        from paper_2208_13770_gb300 import scenes
        sizes = scenes.batch_sizes()
        mine = replicas.shard_greedy(sizes, world)[rank]
        t = torch.tensor([float(sum(int(sizes[q]) for q in mine))], dtype=torch.float64)
        dist.all_reduce(t)
        out.put((rank, mx, replicas.replica_seed(100, rank), mine, float(t.item())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_seeds():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [[2.0, 10.0, 0.5]] * 2
    assert got[0][2] != got[1][2]
    from paper_2208_13770_gb300 import scenes
    sizes = scenes.batch_sizes()
    assert sorted(got[0][3] + got[1][3]) == list(range(len(sizes)))
    assert got[0][4] == got[1][4] == float(sizes.sum())


def test_shard_greedy_balances_scenes():
    from paper_2208_13770_gb300 import replicas, scenes
    sizes = scenes.batch_sizes()
    for world in (1, 2, 3, 8):
        shares = replicas.shard_greedy(sizes, world)
        assert sorted(q for s in shares for q in s) == list(range(len(sizes)))
        loads = [int(sum(sizes[q] for q in s)) for s in shares]
        # largest-first greedy: no rank more than the largest scene above another
        assert max(loads) - min(loads) <= int(sizes.max())
        assert all(s == sorted(s) for s in shares)
    assert replicas.shard_greedy([5, 4, 3], 2) == [[0], [1, 2]]


def test_single_rank_identity_and_throughput():
    from paper_2208_13770_gb300 import replicas
    assert replicas.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert replicas.job_throughput(2, 200_000, 1000, 50.0) == 2 * 200_000 * 1000 / 0.05
    assert replicas.rank_info({}) == (0, 1, 0)
