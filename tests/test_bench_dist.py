"""Replica scaling in bench.py (host logic, CPU): with world_size 2 over gloo
every rank gets its own seeds, and the whole-job rate is the units of all
ranks over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    work = bench.Work("crbd64", seed_base=1 + 100000 * rank)
    seconds = 2.0 if rank == 0 else 3.0
    rate, slowest = bench.job_rate(1000.0, seconds, dist, "cpu")
    q.put((rank, work.runs[0]["seed"], rate, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, r0, t0), (_, s1, r1, t1) = got
    assert s0 != s1  # replicas run different seeds
    assert t0 == t1 == 3.0  # slowest rank
    assert r0 == r1 == pytest.approx(2 * 1000.0 / 3.0)


def test_job_rate_single_process():
    import bench

    assert bench.job_rate(500.0, 2.0) == (250.0, 2.0)
