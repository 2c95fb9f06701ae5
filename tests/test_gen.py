"""The seeded generator: determinism, sub-range regeneration, workload shapes."""
import math

import numpy as np

import gen


def test_subrange_regenerates_identically():
    w = gen.scaled(gen.WORKLOADS["day"], 100_000)
    net, ln = gen.make_table(w.table, w.seed)
    full = gen.make_records(w.records, w.seed, net, ln)
    part = gen.make_records(w.records, w.seed, net, ln, first=31_337, n=1000)
    for k in full:
        assert np.array_equal(full[k][31_337:32_337], part[k])


def test_seed_changes_everything():
    w = gen.scaled(gen.WORKLOADS["tiny"], 10_000)
    net, ln = gen.make_table(w.table, w.seed)
    a = gen.make_records(w.records, w.seed, net, ln)
    b = gen.make_records(w.records, w.seed + 1, net, ln)
    assert (a["src"] != b["src"]).mean() > 0.9


def test_class_mix_and_bytes():
    w = gen.scaled(gen.WORKLOADS["tiny"], 200_000)
    net, ln = gen.make_table(w.table, w.seed)
    r = gen.make_records(w.records, w.seed, net, ln, with_class=True)
    frac = np.bincount(r["intended_class"], minlength=4) / len(r["ts"])
    assert np.allclose(frac, [0.1, 0.4, 0.4, 0.1], atol=0.005)
    lb = np.log(np.maximum(r["bytes"].astype(np.float64), 1))
    assert abs(np.median(lb) - 8.0) < 0.05  # log-normal mu = 8
    assert r["ts"].max() < 3_600_000
    assert ln.min() >= 16 and ln.max() <= 24


def test_diurnal_peak_to_trough_and_order():
    w = gen.scaled(gen.WORKLOADS["day"], 2_000_000)
    net, ln = gen.make_table(w.table, w.seed)
    r = gen.make_records(w.records, w.seed, net, ln)
    ts = r["ts"].astype(np.int64)
    hourly = np.bincount(ts // 3_600_000, minlength=24)
    # rate 2 + cos(.): hourly peak/trough close to 3:1, peak near 14:00
    assert 2.8 < hourly.max() / hourly.min() < 3.05
    assert abs(int(np.argmax(hourly)) - 13.5) <= 1
    # sorted up to the +-500 ms jitter
    assert np.all(np.maximum.accumulate(ts) - ts <= 1000)


def test_zipf_top_bin_matches_closed_form():
    s, n = 1.1, gen.DAY_MS
    k = gen.zipf_ranks(s, n, 99, 400_000)
    h = sum(i ** -s for i in range(1, 200_000)) + (200_000 ** (1 - s) - n ** (1 - s)) / (s - 1)
    p1 = 1.0 / h  # P(rank 1)
    assert abs((k == 1).mean() - p1) < 0.003
    assert abs((k == 2).mean() - p1 * 2 ** -s) < 0.003
    assert k.min() >= 1 and k.max() <= n


def test_batch_plan_shape():
    sl = gen.batch_slices()
    assert len(sl) == 256
    ns = np.array([s.n for s in sl])
    assert ns.min() >= 10_000 and ns.max() <= 20_000_000
    assert 3e8 < ns.sum() < 1.2e9
    assert {s.bin_width for s in sl} <= {1, 10, 1000}
    for s in sl:
        assert 60_000 <= s.window <= 21_600_000
        assert s.n_bins == math.ceil(s.window / s.bin_width)
        assert 16 <= s.table.n <= 4000
