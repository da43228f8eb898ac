"""The multi-rank bench path (replicas, weak scaling) on CPU: two gloo ranks
take the slowest rank's time, agree on the whole-job rate, and draw
disjoint instances."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + rank, world)          # rank 1 is the slower one
        rate = bench.job_throughput(1000.0, t, world)
        seeds = bench.replica_seeds(rank, 3)
        out.put((rank, t, rate, seeds))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, t0, r0, s0), (_, t1, r1, s1) = res
    assert t0 == t1 == 2.0
    assert r0 == r1 == 2 * 1000.0 / 2.0
    assert not set(s0) & set(s1)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(10.0, 2.0, 1) == 5.0
