"""The multi-rank bench path on CPU: two gloo ranks (127.0.0.1) agree on the
slowest rank's time, the whole-job rate counts every rank's units over that
time, and every rank draws its own workload."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import gen

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank  # this rank's timed region, ms
        slowest = bench.max_over_ranks(mine, torch.device("cpu"))
        rate = bench.job_rate(1_000_000, world, 4, slowest)
        w = gen.scaled(gen.WORKLOADS["tiny"], 1000)
        net, ln = gen.make_table(w.table, w.seed)
        rec = gen.make_records(w.records, bench.rank_seed(w.seed, rank), net, ln)
        dist.barrier()
        q.put((rank, slowest, rate, bench.dist_env(), int(rec["ts"][:64].sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_shards():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, slowest, rate, env, _ in got:
        assert slowest == 15.0  # both ranks see the slowest rank's time
        assert rate == pytest.approx(2 * 1_000_000 * 4 / 0.015)
        assert env == (rank, world, rank)
    assert got[0][4] != got[1][4]  # different workloads per rank (weak scaling)


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.job_rate(10, 1, 2, 1000.0) == 20.0
