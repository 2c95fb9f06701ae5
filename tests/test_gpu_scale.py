"""Element-by-element parity against the oracle at sizes where the kernels'
contention and page/bucket machinery are exercised for real:

- config 1 at its stated size (1,000,000 records, 64 prefixes, 3.6 M one-ms
  bins), every strategy that runs it;
- a heavy-shaped day (Zipf(1.1) bins over 86.4 M one-ms bins and Zipf hosts)
  of 50 M records with a 64-prefix table, so the oracle's every-entry loop
  stays cheap: the hottest bin holds about 5 M records. Every bin is
  compared, the hottest included, plus the per-direction totals of counts
  and byte sums (an invariant that needs no binning).
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np
import pytest

import gen
from helpers import assert_hist_equal, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2106_12863_gb300 as sinet  # noqa: E402

ALL = ["global_atomic", "atomic_noagg", "atomic_cell", "priv_tile", "owner", "sort_reduce", "partition"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    sinet.load()
    yield
    torch.cuda.synchronize()
    assert sinet.sinet_device_status() == 0


@pytest.fixture(scope="module")
def config1(orc):
    w = gen.WORKLOADS["tiny"]
    assert w.records.n == 1_000_000 and w.table.n == 64 and w.n_bins == 3_600_000
    net, ln = gen.make_table(w.table, w.seed)
    rec = gen.make_records(w.records, w.seed, net, ln)
    ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    return w, net, ln, rec, ref


@pytest.mark.parametrize("strategy", ALL)
def test_config1_stated_size(config1, strategy):
    w, net, ln, rec, ref = config1
    out = sinet.Histogram(w.n_bins)
    d = to_dev(rec)
    sinet.discriminate_histogram(sinet.PrefixTable(net, ln), d["ts"], d["src"], d["dst"], d["bytes"],
                                 sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=strategy), out)
    torch.cuda.synchronize()
    assert_hist_equal(out.to_numpy(), ref, f"config 1 {strategy}")


@pytest.fixture(scope="module")
def heavy50(orc):
    w = gen.WORKLOADS["heavy"]
    w = replace(w, table=replace(w.table, n=64), records=replace(w.records, n=50_000_000))
    net, ln = gen.make_table(w.table, w.seed)
    rec = gen.make_records(w.records, w.seed, net, ln)
    ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    tot = ref["count"][0].astype(np.uint64) + ref["count"][1]
    assert tot.max() > 4_000_000  # the Zipf head: one bin holds millions of records
    # totals per direction without binning: one bin spanning the whole window
    whole = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width * w.n_bins, 1)
    return w, net, ln, rec, ref, whole


@pytest.mark.parametrize("strategy", ["atomic_cell", "global_atomic", "sort_reduce", "partition"])
def test_heavy_shaped_50M_every_bin(heavy50, strategy):
    w, net, ln, rec, ref, whole = heavy50
    d = to_dev(rec)
    out = sinet.Histogram(w.n_bins, zero=False)
    out.count.fill_(-1)
    out.bytes.fill_(-1)
    sinet.discriminate_histogram(sinet.PrefixTable(net, ln), d["ts"], d["src"], d["dst"], d["bytes"],
                                 sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=strategy), out)
    torch.cuda.synchronize()
    got = out.to_numpy()
    del d, out
    for dd in (0, 1):
        assert int(got["count"][dd].astype(np.uint64).sum()) == int(whole["count"][dd][0])
        assert int(got["bytes"][dd].sum(dtype=np.uint64)) == int(whole["bytes"][dd][0])
    assert_hist_equal(got, ref, f"heavy 50M {strategy}")
    torch.cuda.empty_cache()
