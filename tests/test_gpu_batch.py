"""GPU parity of the batched persistent launch: every slice of a batch
against the oracle run on that slice alone, element by element, bit-exact;
graph replays; accumulating slices; empty, unaligned and out-of-window
slices; every update scheme and lookup form; the autotuner and its cache."""
from __future__ import annotations

import numpy as np
import pytest

import gen
from helpers import assert_hist_equal, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2106_12863_gb300 as sinet  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    sinet.load()
    yield
    torch.cuda.synchronize()
    assert sinet.sinet_device_status() == 0


def _dense80():
    net = np.array([0x0A000000 + 7 * i for i in range(80)], np.uint32)
    return net, np.full(80, 32, np.uint8)


class Case:
    """One slice: host records and table, device tensors, params, outputs."""

    def __init__(self, net, ln, rec, t0, w, n_bins, policy=sinet.EXCLUSIVE, strategy="auto",
                 accumulate=False, offsets=None):
        self.net, self.ln, self.rec = net, ln, rec
        self.t0, self.w, self.n_bins, self.policy = t0, w, n_bins, policy
        self.table = sinet.PrefixTable(net, ln)
        self.dev = to_dev(rec, offsets=offsets)
        self.params = sinet.HistParams(t0, w, n_bins, policy=policy, strategy=strategy,
                                       accumulate=accumulate)
        self.out = sinet.Histogram(n_bins, zero=False)
        self.accumulate = accumulate
        if accumulate:  # start from a known non-zero histogram
            rng = np.random.default_rng(n_bins)
            self.pre = {"count": rng.integers(0, 2 ** 32, (2, n_bins), dtype=np.uint64).astype(np.uint32),
                        "bytes": rng.integers(0, 2 ** 62, (2, n_bins), dtype=np.uint64),
                        "stats": rng.integers(0, 2 ** 40, 8, dtype=np.uint64)}
            self.out.count.copy_(torch.from_numpy(self.pre["count"].view(np.int32)))
            self.out.bytes.copy_(torch.from_numpy(self.pre["bytes"].view(np.int64)))
            self.out.stats.copy_(torch.from_numpy(self.pre["stats"].view(np.int64)))
        else:  # garbage the launch must overwrite
            self.out.count.fill_(-1)
            self.out.bytes.fill_(-1)
            self.out.stats.fill_(-1)

    def slice(self):
        d = self.dev
        return (self.table, d["ts"], d["src"], d["dst"], d["bytes"], self.params, self.out)

    def want(self, orc, runs=1):
        ref = orc.discriminate_histogram(self.net, self.ln, self.rec, self.t0, self.w, self.n_bins,
                                         self.policy)
        if not self.accumulate:
            return ref
        with np.errstate(over="ignore"):
            return {k: self.pre[k] + ref[k] * np.array(runs, ref[k].dtype) for k in ref}


def _generated(n_slices, scale, strategies):
    cases = []
    for i, sp in enumerate(gen.batch_slices(n_slices=n_slices, scale=scale)):
        net, ln = gen.make_table(sp.table, sp.seed)
        rec = gen.make_records(sp.records, sp.seed, net, ln)
        strat = strategies[i % len(strategies)]
        if strat == "smem_full" and sp.n_bins > 2000:
            strat = "auto"
        cases.append(Case(net, ln, rec, sp.t0, sp.bin_width, sp.n_bins, strategy=strat))
    return cases


def _edge_cases():
    w = gen.WORKLOADS["tiny"]
    net, ln = gen.make_table(w.table, w.seed)
    cases = []
    # one slice over many work items with a small histogram (the tile scheme)
    r = gen.make_records(gen.scaled(w, 1_000_003).records, w.seed + 1, net, ln)
    r["ts"] = (r["ts"] % 3_000_000).astype(np.uint64)
    cases.append(Case(net, ln, r, 0, 1000, 3000, policy=sinet.INCLUSIVE, strategy="smem_full"))
    # the same records, plain atomics, paper's literal policy, part of the day outside the window
    cases.append(Case(net, ln, r, 500_000, 1000, 1700, policy=sinet.PAPER_ALG1, strategy="atomic_noagg"))
    # empty slice: its outputs are still zeroed
    e = {k: v[:0] for k, v in r.items()}
    cases.append(Case(net, ln, e, 0, 1, 100, strategy="global_atomic"))
    # unaligned streams and a ragged length
    u = {k: v[:77_777] for k, v in r.items()}
    cases.append(Case(net, ln, u, 0, 7, 500_000, strategy="global_atomic",
                      offsets={"ts": 1, "src": 3, "dst": 2, "bytes": 1}))
    # a table too dense for the shared-memory form (global interval lookups)
    dn, dl = _dense80()
    g = gen.make_records(gen.scaled(w, 300_001).records, w.seed + 2, dn, dl)
    cases.append(Case(dn, dl, g, 0, 1, 3_600_000, strategy="global_atomic"))
    cases.append(Case(dn, dl, g, 0, 10, 360_000, strategy="atomic_noagg"))
    cases.append(Case(dn, dl, g, 0, 1000, 3600, strategy="smem_full"))
    # accumulating into an existing histogram, tile scheme and atomics
    cases.append(Case(net, ln, u, 0, 2000, 1800, strategy="smem_full", accumulate=True))
    cases.append(Case(net, ln, u, 0, 1, 3_600_000, strategy="global_atomic", accumulate=True))
    # the plain path as a chain of its own in the batch's graph: zeroed, and
    # accumulating, with the inclusive policy (two directions per record)
    cases.append(Case(net, ln, r, 0, 1, 3_600_000, policy=sinet.INCLUSIVE, strategy="sort_reduce"))
    cases.append(Case(net, ln, u, 0, 10, 360_000, strategy="sort_reduce", accumulate=True))
    return cases


def _check(orc, cases, runs=1):
    for i, c in enumerate(cases):
        assert_hist_equal(c.out.to_numpy(), c.want(orc, runs), f"slice {i}")


def test_batch_parity_and_replay(orc):
    cases = _generated(32, 0.01, ["auto", "global_atomic", "atomic_noagg", "smem_full", "sort_reduce"]) + _edge_cases()
    b = sinet.Batch([c.slice() for c in cases])
    items, records = b.info()
    assert records == sum(len(c.rec["ts"]) for c in cases)
    assert items >= len(cases) - 1
    for i, c in enumerate(cases):
        s = b.strategy(i)
        assert s in ("global_atomic", "atomic_noagg", "smem_full", "sort_reduce")
        if c.params.strategy != "auto":
            assert s == c.params.strategy
    b.run()
    torch.cuda.synchronize()
    _check(orc, cases, 1)
    b.run()  # graph replay: zeroed slices give the same result, accumulating ones add again
    torch.cuda.synchronize()
    _check(orc, cases, 2)
    b.close()


def test_batch_matches_single_slice_calls(orc):
    """The batch gives what one sinet_discriminate_histogram call per slice gives."""
    cases = _generated(12, 0.02, ["global_atomic", "atomic_noagg"])
    b = sinet.Batch([c.slice() for c in cases])
    b.run()
    torch.cuda.synchronize()
    for i, c in enumerate(cases):
        one = sinet.Histogram(c.n_bins)
        d = c.dev
        sinet.discriminate_histogram(c.table, d["ts"], d["src"], d["dst"], d["bytes"],
                                     sinet.HistParams(c.t0, c.w, c.n_bins, policy=c.policy), one)
        torch.cuda.synchronize()
        assert_hist_equal(c.out.to_numpy(), one.to_numpy(), f"slice {i}")
    b.close()


def test_batch_autotune_and_cache(orc, tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("SINET_AUTOTUNE_CACHE", str(path))
    cases = _generated(20, 0.05, ["auto"])
    b = sinet.Batch([c.slice() for c in cases], autotune=True)
    lines = path.read_text().splitlines() if path.exists() else []
    for ln_ in lines:
        key, name, ms = ln_.split()
        assert key.startswith("sm") and name in ("global_atomic", "atomic_noagg", "smem_full", "sort_reduce")
        assert float(ms) > 0
    b.run()
    torch.cuda.synchronize()
    _check(orc, cases, 1)
    # tuned classes are cached: a second batch of the same shapes tunes nothing new
    n_before = len(lines)
    b2 = sinet.Batch([c.slice() for c in cases], autotune=True)
    lines2 = path.read_text().splitlines() if path.exists() else []
    assert len(lines2) == n_before
    for i in range(len(cases)):
        assert b2.strategy(i) == b.strategy(i)
    b.close()
    b2.close()


def test_batch_ready_word_timeout(orc):
    """A slice whose ready word is never set: its items wait out the bound,
    are left out, and the device status says SINET_ERR_TIMEOUT; the other
    slices are exact."""
    cases = _generated(3, 0.005, ["global_atomic", "atomic_noagg", "smem_full"])
    word = torch.zeros(4, dtype=torch.int32, device="cuda")
    b = sinet.Batch([c.slice() for c in cases], ready=[None, (word[0:1], 1), None])
    b.set_wait(2_000_000)  # 2 ms
    b.run()
    torch.cuda.synchronize()
    assert sinet.sinet_device_status() == 5  # SINET_ERR_TIMEOUT, now cleared
    for i in (0, 2):
        assert_hist_equal(cases[i].out.to_numpy(), cases[i].want(orc), f"slice {i}")
    left = cases[1].out.to_numpy()
    assert not left["count"].any() and not left["bytes"].any()  # zeroed, never filled
    b.close()


def test_batch_ready_word_set_by_a_copy_on_another_stream(orc):
    """The launch starts before a copy on another stream has filled a slice's
    records; the slice's items wait for the ready word the copy stream writes
    after the records and then see the copied records."""
    cases = _generated(4, 0.01, ["global_atomic", "atomic_noagg", "auto", "auto"])
    target = cases[2]
    real = {k: v.clone() for k, v in target.dev.items()}
    for v in target.dev.values():
        v.zero_()  # the launch must not see these
    host = {k: v.cpu().pin_memory() for k, v in real.items()}
    word = torch.zeros(1, dtype=torch.int32, device="cuda")
    seven = torch.full((1,), 7, dtype=torch.int32).pin_memory()
    b = sinet.Batch([c.slice() for c in cases], ready=[None, None, (word, 7), None])
    side = torch.cuda.Stream()
    filler = torch.empty(1 << 28, dtype=torch.uint8).pin_memory()  # 256 MB ahead of the records
    filler_dev = torch.empty_like(filler, device="cuda")
    b.run()  # on the current stream
    with torch.cuda.stream(side):
        filler_dev.copy_(filler, non_blocking=True)
        for k, v in target.dev.items():
            v.copy_(host[k], non_blocking=True)
        word.copy_(seven, non_blocking=True)
    torch.cuda.synchronize()
    assert sinet.sinet_device_status() == 0
    for i, c in enumerate(cases):
        assert_hist_equal(c.out.to_numpy(), c.want(orc), f"slice {i}")
    b.close()


def test_batch_more_slices_than_shared_starts(orc):
    """Over 1,024 slices the work-item starts are searched in global memory
    instead of shared memory; every slice still matches the oracle."""
    w = gen.WORKLOADS["tiny"]
    net, ln = gen.make_table(w.table, w.seed)
    rec = gen.make_records(gen.scaled(w, 1_500 * 700).records, w.seed + 7, net, ln)
    table = sinet.PrefixTable(net, ln)
    dev = to_dev(rec)
    slices, outs, spans = [], [], []
    rng = np.random.default_rng(5)
    for i in range(1_500):
        a, b_ = 700 * i, 700 * i + int(rng.integers(0, 701))  # 0..700 records, some empty
        nb = int(rng.integers(1, 5000))
        bw = int(rng.choice([1, 10, 1000]))
        out = sinet.Histogram(nb, zero=False)
        outs.append(out)
        spans.append((a, b_, nb, bw))
        slices.append((table, dev["ts"][a:b_], dev["src"][a:b_], dev["dst"][a:b_], dev["bytes"][a:b_],
                       sinet.HistParams(0, bw, nb, strategy=("global_atomic", "atomic_noagg", "auto")[i % 3]), out))
    batch = sinet.Batch(slices)
    batch.run()
    torch.cuda.synchronize()
    for i, (a, b_, nb, bw) in enumerate(spans):
        part = {k: v[a:b_] for k, v in rec.items()}
        assert_hist_equal(outs[i].to_numpy(), orc.discriminate_histogram(net, ln, part, 0, bw, nb), f"slice {i}")
    batch.close()
