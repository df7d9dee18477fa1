"""The multi-GPU path on CPU: world size 2 over gloo (127.0.0.1).

Each rank runs its own seeded replica; the job's time is the maximum over
the ranks and its throughput counts every rank's particle-steps.  Here each
rank reports a different time; both must see the same maxima, and the
replica seeds must differ by rank.
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
        out.put((rank, mx, replicas.replica_seed(100, rank)))
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


def test_single_rank_identity_and_throughput():
    from paper_2208_13770_gb300 import replicas
    assert replicas.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert replicas.job_throughput(2, 200_000, 1000, 50.0) == 2 * 200_000 * 1000 / 0.05
    assert replicas.rank_info({}) == (0, 1, 0)
