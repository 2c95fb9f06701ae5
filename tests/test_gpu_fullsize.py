"""Full-size parity at the benchmark's sizes and launch configurations: the
day workload (400 M time-sorted records, 86.4 M bins) with the tile and
owner-computes strategies, the heavy workload (1.6 B unsorted Zipf records) with the
cell and hot/cold partition strategies (the two the benchmark's tuning picks
between), and the 256-slice batch (708 M records) with
the autotuner's choices. The oracle recomputes a sample of bins one by one
(it scans every record and keeps only those bins): random bins, the window's
edges and the hottest bins. Every output also meets the invariants that hold
at any size, and two independent update schemes agree on every element."""
from __future__ import annotations

import numpy as np
import pytest

import gen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def _pinned(w, seed=None):
    n = w.records.n
    net, ln = gen.make_table(w.table, w.seed)
    h = {"ts": torch.empty(n, dtype=torch.int64, pin_memory=True),
         "src": torch.empty(n, dtype=torch.int32, pin_memory=True),
         "dst": torch.empty(n, dtype=torch.int32, pin_memory=True),
         "bytes": torch.empty(n, dtype=torch.int32, pin_memory=True)}
    gen.fill_records(w.records, w.seed if seed is None else seed, net, ln, 0, n, h["ts"], h["src"],
                     h["dst"], h["bytes"])
    return net, ln, h


def _host_view(h):
    return {"ts": h["ts"].numpy().view(np.uint64), "src": h["src"].numpy().view(np.uint32),
            "dst": h["dst"].numpy().view(np.uint32), "bytes": h["bytes"].numpy().view(np.uint32)}


def _sample(count, n_bins, seed, k=3000, hot=(0, 500)):
    """Random bins, the window's edges, and the bins of hotness rank
    hot[0] .. hot[1] - 1 (the oracle classifies every record in a kept bin, so
    under Zipf bins the very hottest are left to the invariants)."""
    rng = np.random.default_rng(seed)
    tot = count[0].astype(np.uint64) + count[1]
    order = np.argsort(tot)[::-1]
    keep = np.concatenate([rng.integers(0, n_bins, k), order[hot[0]:hot[1]], [0, n_bins - 1]])
    return np.unique(keep).astype(np.uint64)


def _invariants(got, n, policy):
    st = got["stats"]
    assert int(st[:4].sum()) == n, "every record is classified once"
    for d in (0, 1):
        routed = sum(int(st[c]) for c in range(4) if policy[c] >> d & 1)
        assert int(got["count"][d].astype(np.uint64).sum()) + int(st[4 + d]) == routed


def _check_sampled(orc, net, ln, rec, w, got, policy, seed, hot):
    keep = _sample(got["count"], w.n_bins, seed, hot=hot)
    c, b = orc.histogram_bins(net, ln, rec, w.t0, w.bin_width, w.n_bins, keep, policy)
    idx = keep.astype(np.int64)
    assert np.array_equal(c, got["count"][:, idx]), "sampled counts differ from the oracle"
    assert np.array_equal(b, got["bytes"][:, idx]), "sampled byte sums differ from the oracle"


@pytest.mark.parametrize("key,strategy,other,hot", [("day", "priv_tile", "global_atomic", (0, 500)),
                                                    ("day", "owner", "priv_tile", (0, 500)),
                                                    ("heavy", "atomic_cell", "global_atomic", (1000, 1020)),
                                                    ("heavy", "partition", "atomic_cell", (1000, 1020))])
def test_full_workload(orc, key, strategy, other, hot):
    w = gen.WORKLOADS[key]
    net, ln, h = _pinned(w)
    d = {k: v.cuda() for k, v in h.items()}
    table = sinet.PrefixTable(net, ln)
    hints = sinet.HINT_TIME_SORTED if w.records.ts_kind == "diurnal" else 0
    out = sinet.Histogram(w.n_bins)
    sinet.discriminate_histogram(table, d["ts"], d["src"], d["dst"], d["bytes"],
                                 sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=strategy,
                                                  hints=hints), out)
    torch.cuda.synchronize()
    got = out.to_numpy()
    _invariants(got, w.records.n, sinet.EXCLUSIVE)
    _check_sampled(orc, net, ln, _host_view(h), w, got, sinet.EXCLUSIVE, 11, hot)
    # an independent update scheme over the same records: equal everywhere
    sinet.discriminate_histogram(table, d["ts"], d["src"], d["dst"], d["bytes"],
                                 sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=other), out)
    torch.cuda.synchronize()
    got2 = out.to_numpy()
    for k in ("stats", "count", "bytes"):
        assert np.array_equal(got[k], got2[k]), f"{strategy} and {other} differ in {k}"
    table.close()
    del d, out
    torch.cuda.empty_cache()


def test_full_batch(orc):
    plan = gen.batch_slices()
    n_tot = sum(sp.n for sp in plan)
    cases, off = [], 0
    h = {"ts": torch.empty(n_tot, dtype=torch.int64, pin_memory=True),
         "src": torch.empty(n_tot, dtype=torch.int32, pin_memory=True),
         "dst": torch.empty(n_tot, dtype=torch.int32, pin_memory=True),
         "bytes": torch.empty(n_tot, dtype=torch.int32, pin_memory=True)}
    for sp in plan:
        net, ln = gen.make_table(sp.table, sp.seed)
        sl = {k: v[off:off + sp.n] for k, v in h.items()}
        gen.fill_records(sp.records, sp.seed, net, ln, 0, sp.n, sl["ts"], sl["src"], sl["dst"], sl["bytes"])
        cases.append((sp, net, ln, off))
        off += sp.n
    d = {k: v.cuda() for k, v in h.items()}
    slices, outs, tabs = [], [], []
    for sp, net, ln, o in cases:
        t = sinet.PrefixTable(net, ln)
        out = sinet.Histogram(sp.n_bins, zero=False)
        tabs.append(t)
        outs.append(out)
        slices.append((t, d["ts"][o:o + sp.n], d["src"][o:o + sp.n], d["dst"][o:o + sp.n],
                       d["bytes"][o:o + sp.n], sinet.HistParams(sp.t0, sp.bin_width, sp.n_bins), out))
    b = sinet.Batch(slices, autotune=True)
    b.run()
    torch.cuda.synchronize()
    hv = _host_view(h)
    for i, (sp, net, ln, o) in enumerate(cases):
        got = outs[i].to_numpy()
        _invariants(got, sp.n, sinet.EXCLUSIVE)
        rec = {k: v[o:o + sp.n] for k, v in hv.items()}
        # about 200 K records' worth of bins per slice (records are uniform over the window)
        k = int(max(2, min(250, 200_000 * sp.n_bins // max(sp.n, 1))))
        keep = _sample(got["count"], sp.n_bins, i, k=k, hot=(0, min(8, k)))
        c, bb = orc.histogram_bins(net, ln, rec, sp.t0, sp.bin_width, sp.n_bins, keep, sinet.EXCLUSIVE)
        idx = keep.astype(np.int64)
        assert np.array_equal(c, got["count"][:, idx]), f"slice {i} counts"
        assert np.array_equal(bb, got["bytes"][:, idx]), f"slice {i} bytes"
    b.close()
