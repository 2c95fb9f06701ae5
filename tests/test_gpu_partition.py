"""GPU parity of the hot/cold partitioned update (SINET_STRAT_PARTITION)
against the oracle, on the paths the generic strategy tests do not reach:
buckets that fill many pages per CTA (beyond the CTA's own page region),
outputs that start as garbage (every bin is stored once), bucket sizes set by
tile_bins, unaligned streams with whole TMA stages, the two-direction policy,
and the refused combinations.
"""
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


def _run(table, dev, params, garbage=True):
    out = sinet.Histogram(params.n_bins, "cuda", zero=not garbage)
    if garbage:  # every bin must be stored by the scheme itself
        out.count.fill_(-7)
        out.bytes.fill_(0x5A5A5A5A5A5A)
        out.stats.fill_(3)
    sinet.discriminate_histogram(table, dev["ts"], dev["src"], dev["dst"], dev["bytes"], params, out)
    torch.cuda.synchronize()
    return out.to_numpy()


def _uniform(n, n_bins, seed, t0=0, width=1):
    w = gen.scaled(gen.WORKLOADS["tiny"], n)
    net, ln = gen.make_table(w.table, w.seed + seed)
    rec = gen.make_records(w.records, w.seed + seed, net, ln)
    rng = np.random.default_rng(seed)
    rec["ts"] = (np.uint64(t0) + rng.integers(0, n_bins * width, n, dtype=np.uint64)).astype(np.uint64)
    return net, ln, rec


@pytest.mark.parametrize("n,n_bins,tile_bins", [
    (3_000_001, 524_288, 0),          # one bucket, ~99 % cold: several pages per CTA
    (8_000_003, 524_288, 0),          # one bucket: each CTA's region overflows into pages taken on demand
    (2_500_003, 3_000_000, 1 << 16),  # 46 buckets of 2^16 bins
    (1_200_007, 40_000_000, 1 << 20), # 39 buckets of 2^20 bins (the largest tile)
])
def test_cold_pages_and_buckets(orc, n, n_bins, tile_bins):
    net, ln, rec = _uniform(n, n_bins, 5)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, n_bins)
    got = _run(sinet.PrefixTable(net, ln), to_dev(rec),
               sinet.HistParams(0, 1, n_bins, strategy="partition", tile_bins=tile_bins))
    assert_hist_equal(got, ref, f"n={n} bins={n_bins} tile={tile_bins}")


@pytest.mark.parametrize("policy", ["inclusive", "paper_alg1"])
def test_two_directions_and_width(orc, policy):
    pol = {"inclusive": sinet.INCLUSIVE, "paper_alg1": sinet.PAPER_ALG1}[policy]
    w = gen.scaled(gen.WORKLOADS["heavy"], 1_000_003)
    net, ln = gen.make_table(w.table, w.seed)
    rec = gen.make_records(w.records, w.seed, net, ln)
    # width 7 ms over the day: a divided bin, hot Zipf bins spread by the division
    ref = orc.discriminate_histogram(net, ln, rec, 3, 7, gen.DAY_MS // 7, pol)
    got = _run(sinet.PrefixTable(net, ln), to_dev(rec),
               sinet.HistParams(3, 7, gen.DAY_MS // 7, policy=pol, strategy="partition"))
    assert_hist_equal(got, ref, policy)


@pytest.mark.parametrize("offsets", [{"ts": 1, "src": 1, "dst": 1, "bytes": 1},
                                     {"ts": 1, "src": 3, "dst": 0, "bytes": 2}])
def test_unaligned_whole_stages(orc, offsets):
    # > 1,024 records after the aligned start (whole TMA stages), or none
    # staged when no common aligned start exists
    net, ln, rec = _uniform(700_001, 2_000_000, 9)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, 2_000_000)
    got = _run(sinet.PrefixTable(net, ln), to_dev(rec, offsets=offsets),
               sinet.HistParams(0, 1, 2_000_000, strategy="partition"))
    assert_hist_equal(got, ref, str(offsets))


# 1,000,000 bins: every output row 16-byte aligned (vector stores); 999,999:
# the second direction's rows are not (scalar stores)
@pytest.mark.parametrize("n_bins", [1_000_000, 999_999])
def test_accumulate_onto_previous(orc, n_bins):
    net, ln, rec = _uniform(900_001, n_bins, 13)
    t, d = sinet.PrefixTable(net, ln), to_dev(rec)
    p = sinet.HistParams(0, 1, n_bins, strategy="partition")
    out = sinet.Histogram(n_bins, "cuda")
    sinet.discriminate_histogram(t, d["ts"], d["src"], d["dst"], d["bytes"], p, out)
    p.accumulate = True
    sinet.discriminate_histogram(t, d["ts"], d["src"], d["dst"], d["bytes"], p, out)
    torch.cuda.synchronize()
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, n_bins)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, n_bins, into=ref)
    assert_hist_equal(out.to_numpy(), ref, f"accumulate, {n_bins} bins")


def test_refused_combinations():
    net, ln, rec = _uniform(10_000, 1000, 1)
    t, d = sinet.PrefixTable(net, ln), to_dev(rec)
    out = sinet.Histogram(300_000_000 // 1000, "cuda")
    cases = [
        # more bins than 256 ranges of 2^20
        (sinet.HistParams(0, 1, 300_000_000, strategy="partition"), 8),
        # a range of more than 2^20 bins
        (sinet.HistParams(0, 1, 1000, strategy="partition", tile_bins=1 << 21), 8),
        # not a power of two
        (sinet.HistParams(0, 1, 1000, strategy="partition", tile_bins=3000), 1),
    ]
    for p, status in cases:
        o = out if p.n_bins <= 300_000 else sinet.Histogram(p.n_bins, "cuda")
        with pytest.raises(sinet.SinetError) as e:
            sinet.discriminate_histogram(t, d["ts"], d["src"], d["dst"], d["bytes"], p, o)
        assert e.value.status == status
        del o


def test_hot_bins_sharing_a_replicated_set(orc):
    # two very hot bins whose hot-table set is the same (the top 12 bits of
    # bin * 0x9E3779B1 agree, so they share a set for every table size up to
    # 2^12 sets): the hotter takes all four ways, the other one of its copies
    n_bins, n = 524_288, 2_000_003
    net, ln, rec = _uniform(n, n_bins, 13)
    top = lambda b: ((b * 0x9E3779B1) & 0xFFFFFFFF) >> 20
    a = 1234
    b = next(x for x in range(n_bins) if x != a and top(x) == top(a))
    u = np.random.default_rng(13).random(n)
    ts = rec["ts"].copy()
    ts[u < 0.4] = a
    ts[(u >= 0.4) & (u < 0.6)] = b
    rec["ts"] = ts.astype(np.uint64)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, n_bins)
    got = _run(sinet.PrefixTable(net, ln), to_dev(rec), sinet.HistParams(0, 1, n_bins, strategy="partition"))
    assert_hist_equal(got, ref, "two hot bins in one set")
