"""One workload split over two gloo ranks on CPU (127.0.0.1), merged with the
library's sharding helpers, equals the single-rank oracle on every element.

The per-rank compute here is the oracle (there is no GPU in this test); what
is under test is the host side of the multi-GPU path: the record-range and
time-range splits, and the merge collectives (all-reduce, reduce-scatter,
gather of owned slices) with uint32 counts and uint64 byte sums carried bit
for bit, including wrap-around."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _as_torch(h):
    return (torch.from_numpy(h["count"].view(np.int32).copy()),
            torch.from_numpy(h["bytes"].view(np.int64).copy()),
            torch.from_numpy(h["stats"].view(np.int64).copy()))


def _rank_main(rank: int, world: int, port: int, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import gen
    import oracle
    from paper_2106_12863_gb300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        orc = oracle.get()
        w = gen.scaled(gen.WORKLOADS["tiny"], 200_003)
        net, ln = gen.make_table(w.table, w.seed)
        res = {}
        # record-range split: this rank generates only its own records
        lo, hi = shard.record_range(w.records.n, world, rank)
        mine = gen.make_records(w.records, w.seed, net, ln, first=lo, n=hi - lo)
        part = orc.discriminate_histogram(net, ln, mine, w.t0, w.bin_width, w.n_bins)
        if rank == 0:  # a count that wraps modulo 2^32 when merged
            part["count"][0, 5] = np.uint32(0xFFFFFFFF)
        c, b, s = _as_torch(part)
        sc, sb = shard.merge(c.clone(), b.clone(), s.clone(), scatter=True)
        shard.merge(c, b, s)
        res["all"] = (c.numpy().view(np.uint32).copy(), b.numpy().view(np.uint64).copy(),
                      s.numpy().view(np.uint64).copy())
        res["scatter"] = (shard.bin_range(w.n_bins, world, rank), sc.numpy().view(np.uint32).copy(),
                          sb.numpy().view(np.uint64).copy())
        # time-range split: this rank keeps the records of its own bins
        allr = gen.make_records(w.records, w.seed, net, ln)
        win = shard.Window(w.t0, w.bin_width, w.n_bins).owned(world, rank)
        keep = (allr["ts"] >= np.uint64(win.t0)) & (allr["ts"] < np.uint64(win.t0 + win.n_bins * win.width))
        if rank == 0:  # records outside the whole window are counted once, by rank 0
            keep |= (allr["ts"] < np.uint64(w.t0)) | (allr["ts"] >= np.uint64(w.t0 + w.n_bins * w.bin_width))
        own = orc.discriminate_histogram(net, ln, {k: v[keep] for k, v in allr.items()}, win.t0, win.width,
                                         win.n_bins)
        oc, ob, os_ = _as_torch(own)
        fc, fb = shard.gather_owned(oc, ob, os_, w.n_bins)
        res["time"] = (fc.numpy().view(np.uint32).copy(), fb.numpy().view(np.uint64).copy(),
                       os_.numpy().view(np.uint64).copy())
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_sharded_merges_equal_the_single_rank_oracle(orc):
    import gen
    from paper_2106_12863_gb300 import shard

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = gen.scaled(gen.WORKLOADS["tiny"], 200_003)
    net, ln = gen.make_table(w.table, w.seed)
    ref = orc.discriminate_histogram(net, ln, gen.make_records(w.records, w.seed, net, ln),
                                     w.t0, w.bin_width, w.n_bins)
    wrapped = ref["count"].copy()
    wrapped[0, 5] = np.uint32((int(wrapped[0, 5]) + 0xFFFFFFFF) & 0xFFFFFFFF)
    for r in range(world):
        c, b, s = got[r]["all"]
        assert np.array_equal(c, wrapped) and np.array_equal(b, ref["bytes"])
        assert np.array_equal(s, ref["stats"])
        (lo, hi), sc, sb = got[r]["scatter"]
        assert (lo, hi) == shard.bin_range(w.n_bins, world, r)
        assert np.array_equal(sc, wrapped[:, lo:hi]) and np.array_equal(sb, ref["bytes"][:, lo:hi])
        tc, tb, ts = got[r]["time"]
        assert np.array_equal(tc, ref["count"]) and np.array_equal(tb, ref["bytes"])
        assert np.array_equal(ts, ref["stats"])


@pytest.mark.parametrize("n,world", [(0, 3), (1, 2), (10, 4), (1_000_003, 8), (7, 8)])
def test_ranges_partition_the_records_and_bins(n, world):
    from paper_2106_12863_gb300 import shard

    r = [shard.record_range(n, world, k) for k in range(world)]
    assert r[0][0] == 0 and r[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    assert all(lo % 4 == 0 and lo <= hi for lo, hi in r)
    b = [shard.bin_range(n, world, k) for k in range(world)]
    assert b[0][0] == 0 and b[-1][1] == n and all(x[1] == y[0] for x, y in zip(b, b[1:]))
    assert max(hi - lo for lo, hi in b) - min(hi - lo for lo, hi in b) <= 1
