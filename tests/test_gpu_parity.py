"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element, bit-exact (all arithmetic is integer).

Sizes span many CTA tiles and ragged tails; edge cases cover empty and tiny
inputs, unaligned streams, out-of-window records, hot bins, 2^32 - 1 byte
values, accumulation and uint32 wrap-around.
"""
from __future__ import annotations

import random

import numpy as np
import pytest

import gen
import oracle
from helpers import assert_hist_equal, run_fused, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2106_12863_gb300 as sinet  # noqa: E402

STRATS = ["global_atomic", "atomic_noagg", "atomic_cell", "priv_tile", "owner", "sort_reduce", "partition"]
POLICIES = {"exclusive": sinet.EXCLUSIVE, "inclusive": sinet.INCLUSIVE, "paper_alg1": sinet.PAPER_ALG1}


@pytest.fixture(scope="module", autouse=True)
def lib():
    sinet.load()
    yield
    torch.cuda.synchronize()
    assert sinet.sinet_device_status() == 0


def _workload(key, n, seed_shift=0):
    w = gen.scaled(gen.WORKLOADS[key], n)
    net, ln = gen.make_table(w.table, w.seed + seed_shift)
    rec = gen.make_records(w.records, w.seed + seed_shift, net, ln)
    return w, net, ln, rec


def _edge_table(seed):
    rng = random.Random(seed)
    k = 40
    net = np.array([rng.getrandbits(32) for _ in range(k)], np.uint32)
    ln = np.array([rng.choice([0, 1, 8, 12, 16, 20, 24, 28, 31, 32]) for _ in range(k)], np.uint8)
    ln[0] = 3  # no /0 here (it would make everything inside); /0 is covered separately
    ln[ln == 0] = 1
    return net, ln


# ---------------------------------------------------------------------------
# Algorithm 1 alone


def _disc_inputs(net, ln, n, seed):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    dst = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    # plant prefix edges and inside addresses
    m = min(len(net), n // 8)
    for i in range(m):
        z = int(ln[i])
        mask = 0 if z == 0 else (0xFFFFFFFF << (32 - z)) & 0xFFFFFFFF
        lo = int(net[i]) & mask
        hi = lo | (~mask & 0xFFFFFFFF)
        src[8 * i: 8 * i + 4] = [lo, hi, (lo - 1) & 0xFFFFFFFF, (hi + 1) & 0xFFFFFFFF]
        dst[8 * i + 4: 8 * i + 8] = [lo, hi, (lo - 1) & 0xFFFFFFFF, (hi + 1) & 0xFFFFFFFF]
    return src, dst


@pytest.mark.parametrize("lookup", ["interval", "pml"])
@pytest.mark.parametrize("table", ["tiny", "day", "heavy", "edges", "empty", "slash0", "dense", "dense80"])
def test_discriminate_parity(orc, lookup, table):
    if table in gen.WORKLOADS:
        w = gen.WORKLOADS[table]
        net, ln = gen.make_table(w.table, w.seed)
    elif table == "edges":
        net, ln = _edge_table(5)
    elif table == "empty":
        net, ln = np.zeros(0, np.uint32), np.zeros(0, np.uint8)
    elif table in ("dense", "dense80"):  # many /32 hosts in one bucket (variable / global forms)
        k = 20 if table == "dense" else 80
        net = np.array([0x0A000000 + 7 * i for i in range(k)], np.uint32)
        ln = np.full(k, 32, np.uint8)
    else:
        net, ln = np.array([0x0A000000, 0xC0A80000], np.uint32), np.array([0, 16], np.uint8)
    n = 200_003
    src, dst = _disc_inputs(net, ln, n, 7)
    if table in gen.WORKLOADS:  # also real generated records
        w = gen.scaled(gen.WORKLOADS[table], n)
        r = gen.make_records(w.records, w.seed, net, ln)
        src[n // 2:], dst[n // 2:] = r["src"][n // 2:], r["dst"][n // 2:]
    want = orc.classify(net, ln, src, dst) if len(net) else np.zeros(n, np.uint8)
    t = sinet.PrefixTable(net, ln)
    d = to_dev({"src": src, "dst": dst})
    cls = torch.empty(n, dtype=torch.uint8, device="cuda")
    counts = sinet.discriminate(t, d["src"], d["dst"], cls, lookup=lookup)
    torch.cuda.synchronize()
    got = cls.cpu().numpy()
    assert np.array_equal(got, want)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64),
                          np.bincount(want, minlength=4).astype(np.uint64))


@pytest.mark.parametrize("offsets", [{"src": 1, "dst": 1}, {"src": 2, "dst": 1}, {"src": 3, "dst": 3}])
def test_discriminate_unaligned(orc, offsets):
    w = gen.WORKLOADS["day"]
    net, ln = gen.make_table(w.table, w.seed)
    n = 50_001
    src, dst = _disc_inputs(net, ln, n, 3)
    want = orc.classify(net, ln, src, dst)
    t = sinet.PrefixTable(net, ln)
    d = to_dev({"src": src, "dst": dst}, offsets=offsets)
    buf = torch.zeros(n + 3, dtype=torch.uint8, device="cuda")
    cls = buf[1:1 + n]
    counts = sinet.discriminate(t, d["src"], d["dst"], cls)
    torch.cuda.synchronize()
    assert np.array_equal(cls.cpu().numpy(), want)
    assert buf[0].item() == 0 and buf[-2:].sum().item() == 0  # nothing written outside
    assert np.array_equal(counts.cpu().numpy().view(np.uint64),
                          np.bincount(want, minlength=4).astype(np.uint64))


# ---------------------------------------------------------------------------
# fused discriminate + histogram


@pytest.mark.parametrize("lookup", ["interval", "pml"])
@pytest.mark.parametrize("strategy", STRATS)
def test_fused_tiny(orc, strategy, lookup):
    w, net, ln, rec = _workload("tiny", 250_001)
    ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    t = sinet.PrefixTable(net, ln)
    got = run_fused(t, to_dev(rec), sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=strategy,
                                                     lookup=lookup))
    assert_hist_equal(got, ref, f"{strategy}/{lookup}")


@pytest.mark.parametrize("policy", sorted(POLICIES))
@pytest.mark.parametrize("strategy", STRATS + ["smem_full"])
@pytest.mark.parametrize("window", [(500_000, 7, 300_001), (1_000_000, 1000, 1500), (0, 60_000, 61)])
def test_fused_windows_policies(orc, strategy, policy, window):
    t0, wd, nb = window
    if strategy == "smem_full" and nb > 4096:
        pytest.skip("whole-histogram privatisation is for small histograms")
    w, net, ln, rec = _workload("tiny", 120_007, seed_shift=11)
    pol = POLICIES[policy]
    ref = orc.discriminate_histogram(net, ln, rec, t0, wd, nb, pol)
    t = sinet.PrefixTable(net, ln)
    got = run_fused(t, to_dev(rec), sinet.HistParams(t0, wd, nb, policy=pol, strategy=strategy))
    assert_hist_equal(got, ref, f"{strategy}/{policy}/{window}")


@pytest.mark.parametrize("strategy", STRATS)
def test_sorted_day_slice(orc, strategy):
    # a whole day of sorted records (diurnal, +-500 ms jitter), 2 M records
    w, net, ln, rec = _workload("day", 2_000_000)
    ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    t = sinet.PrefixTable(net, ln)
    got = run_fused(t, to_dev(rec), sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=strategy,
                                                     hints=sinet.HINT_TIME_SORTED))
    assert_hist_equal(got, ref, strategy)


@pytest.mark.parametrize("strategy", STRATS)
def test_heavy_zipf_slice(orc, strategy):
    # Zipf(1.1) bins and hosts: ~11% of records in one bin (atomic contention)
    w, net, ln, rec = _workload("heavy", 1_500_003)
    ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    t = sinet.PrefixTable(net, ln)
    got = run_fused(t, to_dev(rec), sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=strategy))
    assert_hist_equal(got, ref, strategy)


def test_histogram_of_classified_records(orc):
    w, net, ln, rec = _workload("tiny", 300_001, seed_shift=2)
    cls = orc.classify(net, ln, rec["src"], rec["dst"])
    d = to_dev({"ts": rec["ts"], "bytes": rec["bytes"], "cls": cls})
    for strategy in STRATS:
        ref = orc.histogram(rec["ts"], rec["bytes"], cls, 1000, 3, 1_000_000, sinet.INCLUSIVE)
        out = sinet.Histogram(1_000_000)
        params = sinet.HistParams(1000, 3, 1_000_000, policy=sinet.INCLUSIVE, strategy=strategy)
        if strategy == "partition":  # fused entry point only
            with pytest.raises(sinet.SinetError) as e:
                sinet.histogram(d["ts"], d["bytes"], d["cls"], params, out)
            assert e.value.status == 8
            continue
        sinet.histogram(d["ts"], d["bytes"], d["cls"], params, out)
        torch.cuda.synchronize()
        assert_hist_equal(out.to_numpy(), ref, strategy)


# ---------------------------------------------------------------------------
# edge cases


def _tiny_rec(n, seed=1):
    w = gen.scaled(gen.WORKLOADS["tiny"], max(n, 1))
    net, ln = gen.make_table(w.table, w.seed)
    rec = gen.make_records(w.records, w.seed + seed, net, ln)
    return w, net, ln, {k: v[:n] for k, v in rec.items()}


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 7, 33, 1023])
@pytest.mark.parametrize("strategy", STRATS)
def test_small_n(orc, n, strategy):
    w, net, ln, rec = _tiny_rec(n)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1000, 3600)
    t = sinet.PrefixTable(net, ln)
    got = run_fused(t, to_dev(rec), sinet.HistParams(0, 1000, 3600, strategy=strategy))
    assert_hist_equal(got, ref, f"n={n}")


@pytest.mark.parametrize("offsets", [{"ts": 1, "src": 1, "dst": 1, "bytes": 1},
                                     {"ts": 2, "src": 2, "dst": 2, "bytes": 2},
                                     {"ts": 1, "src": 3, "dst": 0, "bytes": 2}])
@pytest.mark.parametrize("strategy", STRATS)
def test_unaligned_streams(orc, offsets, strategy):
    w, net, ln, rec = _tiny_rec(40_001)
    ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    t = sinet.PrefixTable(net, ln)
    got = run_fused(t, to_dev(rec, offsets=offsets),
                    sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=strategy))
    assert_hist_equal(got, ref, str(offsets))


@pytest.mark.parametrize("strategy", STRATS + ["smem_full"])
def test_hot_bin_and_max_bytes(orc, strategy):
    w, net, ln, rec = _tiny_rec(100_000)
    rec["ts"][:] = 1234  # every record in one bin
    rec["bytes"][: 50_000] = 0xFFFFFFFF
    ref = orc.discriminate_histogram(net, ln, rec, 1000, 10, 64)
    assert ref["bytes"].max() > 2 ** 40  # sums far above 32 bits
    t = sinet.PrefixTable(net, ln)
    got = run_fused(t, to_dev(rec), sinet.HistParams(1000, 10, 64, strategy=strategy))
    assert_hist_equal(got, ref, strategy)


@pytest.mark.parametrize("strategy", STRATS)
def test_all_out_of_window(orc, strategy):
    w, net, ln, rec = _tiny_rec(10_000)
    ref = orc.discriminate_histogram(net, ln, rec, 10 ** 9, 1, 1000)
    assert ref["count"].sum() == 0
    t = sinet.PrefixTable(net, ln)
    got = run_fused(t, to_dev(rec), sinet.HistParams(10 ** 9, 1, 1000, strategy=strategy))
    assert_hist_equal(got, ref, strategy)


def test_large_t0_and_width(orc):
    w, net, ln, rec = _tiny_rec(20_000)
    base = (1 << 62) + 12345
    rec["ts"] = rec["ts"] * np.uint64(1_000_003) + np.uint64(base)
    for strategy in STRATS:
        ref = orc.discriminate_histogram(net, ln, rec, base, 999_983, 3_700_000)
        t = sinet.PrefixTable(net, ln)
        got = run_fused(t, to_dev(rec), sinet.HistParams(base, 999_983, 3_700_000, strategy=strategy))
        assert_hist_equal(got, ref, strategy)


@pytest.mark.parametrize("strategy", STRATS)
def test_accumulate_and_wrap(orc, strategy):
    w, net, ln, rec = _tiny_rec(60_000)
    t = sinet.PrefixTable(net, ln)
    d = to_dev(rec)
    params = sinet.HistParams(0, 1000, 3600, strategy=strategy)
    out = sinet.Histogram(3600)
    sinet.discriminate_histogram(t, d["ts"], d["src"], d["dst"], d["bytes"], params, out)
    out.count[0, 17] = -1  # 0xFFFFFFFF: the next add wraps
    params.accumulate = True
    sinet.discriminate_histogram(t, d["ts"], d["src"], d["dst"], d["bytes"], params, out)
    torch.cuda.synchronize()
    got = out.to_numpy()
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1000, 3600)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1000, 3600, into=ref)
    single = orc.discriminate_histogram(net, ln, rec, 0, 1000, 3600)
    ref["count"][0, 17] = np.uint32((0xFFFFFFFF + int(single["count"][0, 17])) & 0xFFFFFFFF)
    assert_hist_equal(got, ref, strategy)


def test_device_status_is_clean_after_runs():
    torch.cuda.synchronize()
    assert sinet.sinet_device_status() == 0


# ---------------------------------------------------------------------------
# Watch list: only records with src or dst in a second list are binned


def _watch_list(rec, seed, hosts=300, prefixes=4):
    rng = np.random.default_rng(seed)
    h = np.unique(np.concatenate([rng.choice(rec["src"], hosts // 2), rng.choice(rec["dst"], hosts // 2)]))
    pre = rng.integers(0, 2 ** 32, prefixes, dtype=np.uint64).astype(np.uint32) & np.uint32(0xFFFF0000)
    net = np.concatenate([h, pre]).astype(np.uint32)
    ln = np.concatenate([np.full(len(h), 32, np.uint8), np.full(len(pre), 16, np.uint8)])
    return net, ln


@pytest.mark.parametrize("strategy", ["auto", "global_atomic", "atomic_noagg", "atomic_cell"])
@pytest.mark.parametrize("key", ["tiny", "heavy"])
def test_watch_filter(orc, key, strategy):
    w, net, ln, rec = _workload(key, 400_003)
    wnet, wln = _watch_list(rec, 3)
    want = orc.discriminate_histogram_watch(net, ln, wnet, wln, rec, w.t0, w.bin_width, w.n_bins)
    assert 0 < int(want["stats"][6]) < len(rec["ts"])
    got = run_fused(sinet.PrefixTable(net, ln), to_dev(rec),
                    sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=strategy,
                                     watch=sinet.PrefixTable(wnet, wln)))
    assert_hist_equal(got, want, f"{key} watch {strategy}")


def test_watch_filter_refused_where_not_run(orc):
    w, net, ln, rec = _workload("tiny", 10_000)
    d = to_dev(rec)
    t, wt = sinet.PrefixTable(net, ln), sinet.PrefixTable(*_watch_list(rec, 4))
    out = sinet.Histogram(w.n_bins)
    for s in ("priv_tile", "smem_full", "owner", "sort_reduce", "partition"):
        with pytest.raises(sinet.SinetError) as e:
            sinet.discriminate_histogram(t, d["ts"], d["src"], d["dst"], d["bytes"],
                                         sinet.HistParams(w.t0, w.bin_width, w.n_bins, strategy=s, watch=wt), out)
        assert e.value.status == 8


# ---------------------------------------------------------------------------
# AUTO: the fixed rule, and the measured choice (SINET_HINT_TUNE)


@pytest.mark.parametrize("key,hints", [("heavy", 0), ("day", sinet.HINT_TIME_SORTED), ("tiny", 0)])
def test_auto_measured_choice(orc, key, hints):
    w, net, ln, rec = _workload(key, 600_007)
    ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    t = sinet.PrefixTable(net, ln)
    d = to_dev(rec)
    n = len(rec["ts"])
    p = sinet.HistParams(w.t0, w.bin_width, w.n_bins, hints=hints)
    rule = sinet.auto_strategy(t, n, p)
    assert rule != "auto"
    got = run_fused(t, d, p)
    assert_hist_equal(got, ref, f"auto rule {rule}")
    p.hints = hints | sinet.HINT_TUNE
    first = run_fused(t, d, p)  # times the candidates, then runs the fastest
    assert_hist_equal(first, ref, "auto measured (first call)")
    chosen = sinet.auto_strategy(t, n, p)
    assert chosen in ("smem_full", "priv_tile", "owner", "global_atomic", "atomic_cell", "partition")
    assert sinet.auto_strategy(t, n, sinet.HistParams(w.t0, w.bin_width, w.n_bins, hints=hints)) == chosen
    again = run_fused(t, d, p)  # cached: no timing
    assert_hist_equal(again, ref, f"auto measured (cached {chosen})")


def test_auto_rule_by_input_class():
    # the fixed rule (no kernel runs): the partition for unsorted input over a
    # large histogram with at least one record per four bins, the chunk tile
    # for time-sorted input, warp combining for sparse input
    w = gen.WORKLOADS["heavy"]
    net, ln = gen.make_table(w.table, w.seed)
    t = sinet.PrefixTable(net, ln)
    p = sinet.HistParams(w.t0, w.bin_width, w.n_bins)
    assert sinet.auto_strategy(t, w.records.n, p) == "partition"
    assert sinet.auto_strategy(t, w.records.n, sinet.HistParams(w.t0, w.bin_width, w.n_bins,
                                                                 hints=sinet.HINT_TIME_SORTED)) == "priv_tile"
    assert sinet.auto_strategy(t, w.n_bins // 8, p) == "global_atomic"
    t.close()
