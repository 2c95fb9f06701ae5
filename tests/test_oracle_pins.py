"""Pins for the CPU oracle against things other than itself.

Each check is written as a function of an ``Oracle`` so the same checks can be
run against builds with a planted mistake (``test_planted_mistakes_are_caught``):
every plausible slip in the oracle must fail at least one of them.

Sources of truth used here:
  * hand-worked values (tests/golden/*.txt) for bitmask, membership and a
    whole discriminate + histogram example (Algorithm 1; Section 5);
  * Python's ``ipaddress`` module (a library routine for CIDR membership);
  * brute force over a 12-bit address universe, expanding each prefix into its
    explicit address set by integer division (no masks);
  * ``numpy.bincount`` / ``numpy.add.at`` for the histogram;
  * invariants: class counts sum to N, per-direction totals plus out-of-range
    equal the routed records, additivity over concatenation, order
    independence, uint32 count wrap-around;
  * construction: the generator places "inside" addresses inside a prefix and
    "outside" ones in first octets no prefix uses.
"""
from __future__ import annotations

import ipaddress
import os
import random

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
POLICIES = {"EXCLUSIVE": oracle.EXCLUSIVE, "INCLUSIVE": oracle.INCLUSIVE,
            "PAPER_ALG1": oracle.PAPER_ALG1}


def ip(s: str) -> int:
    return int(ipaddress.IPv4Address(s))


def cidr(s: str):
    a, z = s.split("/")
    return ip(a), int(z)


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


# ---------------------------------------------------------------------------
# checks (each takes an Oracle, raises AssertionError on a mismatch)


def check_bitmask_golden(o):
    for x, z, want in _rows("bitmask_cases.txt"):
        assert o.bitmask(ip(x), int(z)) == ip(want), (x, z, want)


def check_membership_golden(o):
    for a, c, want in _rows("membership_cases.txt"):
        n, z = cidr(c)
        got = o.in_list(ip(a), [n], [z])
        assert got == bool(int(want)), (a, c, want)


def check_membership_ipaddress(o, trials=300, seed=11):
    rng = random.Random(seed)
    for _ in range(trials):
        k = rng.randint(1, 6)
        net = [rng.getrandbits(32) for _ in range(k)]  # host bits left set on purpose
        ln = [rng.choice([0, 1, 7, 8, 12, 16, 20, 24, 25, 30, 31, 32, rng.randint(0, 32)])
              for _ in range(k)]
        nets = [ipaddress.ip_network((n, z), strict=False) for n, z in zip(net, ln)]
        addrs = [rng.getrandbits(32) for _ in range(20)]
        # addresses near the prefix edges too
        for nw in nets:
            lo, hi = int(nw.network_address), int(nw.broadcast_address)
            addrs += [lo, hi, (lo - 1) & 0xFFFFFFFF, (hi + 1) & 0xFFFFFFFF]
        for a in addrs:
            want = any(ipaddress.IPv4Address(a) in nw for nw in nets)
            assert o.in_list(a, net, ln) == want, (a, net, ln)


def _universe_sets(net, ln):
    """Explicit address set of each prefix, by integer division (no masks)."""
    out = set()
    for n, z in zip(net, ln):
        size = 2 ** (32 - z)
        base = (n // size) * size
        out.update(range(base, base + size))
    return out


def check_membership_brute_force(o, trials=60, seed=5):
    rng = random.Random(seed)
    base = ip("10.20.16.0")  # a /20: 4096 addresses
    for _ in range(trials):
        k = rng.randint(0, 8)
        net, ln = [], []
        for _ in range(k):
            z = rng.choice([19, 20, 21, 22, 24, 26, 28, 30, 31, 32, rng.randint(20, 32)])
            n = base + rng.getrandbits(12) if z >= 20 else base + rng.getrandbits(13) - 4096
            net.append(n & 0xFFFFFFFF)
            ln.append(z)
        inside = _universe_sets(net, ln)
        addrs = np.arange(base - 64, base + 4096 + 64, dtype=np.int64)
        cls = o.classify(net if k else [0], ln if k else [0],
                         addrs.astype(np.uint32), np.full(len(addrs), ip("1.1.1.1"), np.uint32)) \
            if k else np.zeros(len(addrs), np.uint8)
        for a, c in zip(addrs.tolist(), cls.tolist()):
            assert bool(c & 1) == (a in inside), (a, net, ln)


def check_class_bits(o):
    net, ln = [ip("10.0.0.0")], [8]
    src = np.array([ip("10.0.0.1"), ip("11.0.0.1"), ip("10.0.0.1"), ip("11.0.0.1")], np.uint32)
    dst = np.array([ip("11.0.0.1"), ip("10.0.0.1"), ip("10.9.0.1"), ip("12.0.0.1")], np.uint32)
    assert o.classify(net, ln, src, dst).tolist() == [1, 2, 3, 0]


def _golden_example():
    table, window, recs, expect = None, None, [], {}
    for row in _rows("histogram_worked_example.txt"):
        if row[0] == "table":
            table = [cidr(c) for c in row[1:]]
        elif row[0] == "window":
            window = tuple(int(v) for v in row[1:])
        elif row[0] == "rec":
            recs.append((int(row[1]), ip(row[2]), ip(row[3]), int(row[4])))
        elif row[0] == "expect":
            expect.setdefault(row[1], {})[row[2]] = [int(v) for v in row[3:]]
    rec = {"ts": np.array([r[0] for r in recs], np.uint64),
           "src": np.array([r[1] for r in recs], np.uint32),
           "dst": np.array([r[2] for r in recs], np.uint32),
           "bytes": np.array([r[3] for r in recs], np.uint32)}
    net = np.array([t[0] for t in table], np.uint32)
    ln = np.array([t[1] for t in table], np.uint8)
    return net, ln, rec, window, expect


def check_histogram_golden(o):
    net, ln, rec, (t0, w, nb), expect = _golden_example()
    for pname, exp in expect.items():
        h = o.discriminate_histogram(net, ln, rec, t0, w, nb, POLICIES[pname])
        assert h["count"][0].tolist() == exp["count_out"], pname
        assert h["bytes"][0].tolist() == exp["bytes_out"], pname
        assert h["count"][1].tolist() == exp["count_in"], pname
        assert h["bytes"][1].tolist() == exp["bytes_in"], pname
        assert h["stats"].tolist() == exp["stats"], pname


def _random_classified(seed, n, n_bins, t0, w):
    rng = np.random.default_rng(seed)
    lo = max(0, t0 - 3 * w)
    ts = rng.integers(lo, t0 + n_bins * w + 3 * w, n, dtype=np.int64).astype(np.uint64)
    nb = rng.integers(0, 2 ** 32, n, dtype=np.int64).astype(np.uint32)
    nb[: n // 50] = 0xFFFFFFFF
    cls = rng.integers(0, 4, n).astype(np.uint8)
    return ts, nb, cls


def check_histogram_numpy(o, seed=3):
    for t0, w, n_bins in ((0, 1, 1000), (1234, 7, 301), (10 ** 12, 1000, 17)):
        ts, nb, cls = _random_classified(seed, 20_000, n_bins, t0, w)
        for policy in POLICIES.values():
            h = o.histogram(ts, nb, cls, t0, w, n_bins, policy)
            tsi = ts.astype(object)
            inr = np.array([(t >= t0) and ((t - t0) // w < n_bins) for t in tsi])
            b = np.array([(t - t0) // w if (t >= t0) else -1 for t in tsi], dtype=np.int64)
            dirs = np.asarray(policy, np.uint8)[cls]
            for d in (0, 1):
                routed = ((dirs >> d) & 1).astype(bool)
                sel = routed & inr
                cnt = np.bincount(b[sel], minlength=n_bins)
                assert np.array_equal(h["count"][d], cnt.astype(np.uint32))
                s = np.zeros(n_bins, np.uint64)
                np.add.at(s, b[sel], nb[sel].astype(np.uint64))
                assert np.array_equal(h["bytes"][d], s)
                assert h["stats"][4 + d] == int((routed & ~inr).sum())
            assert np.array_equal(h["stats"][:4], np.bincount(cls, minlength=4).astype(np.uint64))


def check_brute_force_pipeline(o, seed=17):
    """Pure-Python loops over a tiny workload: sets for membership, ints for bins."""
    rng = random.Random(seed)
    base = ip("10.20.16.0")
    for trial in range(6):
        k = rng.randint(1, 5)
        net = [(base + rng.getrandbits(12)) & 0xFFFFFFFF for _ in range(k)]
        ln = [rng.randint(20, 32) for _ in range(k)]
        inside = _universe_sets(net, ln)
        t0, w, nb = rng.randint(0, 50), rng.randint(1, 5), rng.randint(1, 9)
        recs = []
        for _ in range(150):
            recs.append((rng.randint(0, t0 + w * nb + 10), base + rng.getrandbits(12) - 16,
                         base + rng.getrandbits(12) - 16, rng.getrandbits(32)))
        rec = {"ts": np.array([r[0] for r in recs], np.uint64),
               "src": np.array([r[1] for r in recs], np.uint32),
               "dst": np.array([r[2] for r in recs], np.uint32),
               "bytes": np.array([r[3] for r in recs], np.uint32)}
        for policy in POLICIES.values():
            cnt = [[0] * nb for _ in range(2)]
            byt = [[0] * nb for _ in range(2)]
            stats = [0] * 8
            for ts, s, d, b in recs:
                c = int(s in inside) + 2 * int(d in inside)
                stats[c] += 1
                for di in (0, 1):
                    if policy[c] & (1 << di):
                        if t0 <= ts < t0 + nb * w:
                            cnt[di][(ts - t0) // w] += 1
                            byt[di][(ts - t0) // w] += b
                        else:
                            stats[4 + di] += 1
            h = o.discriminate_histogram(np.array(net, np.uint32), np.array(ln, np.uint8), rec, t0,
                                         w, nb, policy)
            assert h["count"].tolist() == cnt, trial
            assert h["bytes"].tolist() == byt, trial
            assert h["stats"].tolist() == stats, trial


def check_invariants_generated(o, seed=7):
    wl = gen.scaled(gen.WORKLOADS["tiny"], 50_000)
    net, ln = gen.make_table(wl.table, wl.seed + seed)
    rec = gen.make_records(wl.records, wl.seed + seed, net, ln, with_class=True)
    cls = o.classify(net, ln, rec["src"], rec["dst"])
    # construction: inside/outside by construction, so classes are known exactly
    assert np.array_equal(cls, rec["intended_class"])
    for policy in POLICIES.values():
        h = o.discriminate_histogram(net, ln, rec, wl.t0, wl.bin_width, wl.n_bins, policy)
        st = h["stats"]
        assert int(st[:4].sum()) == len(rec["ts"])
        dirs = np.asarray(policy, np.uint8)[cls]
        for d in (0, 1):
            routed = ((dirs >> d) & 1).astype(bool)
            assert int(h["count"][d].sum(dtype=np.uint64)) + int(st[4 + d]) == int(routed.sum())
        # concatenation additivity and order independence
        half = len(rec["ts"]) // 3
        a = {k: v[:half] for k, v in rec.items()}
        b = {k: v[half:] for k, v in rec.items()}
        hab = o.discriminate_histogram(net, ln, a, wl.t0, wl.bin_width, wl.n_bins, policy)
        hab = o.discriminate_histogram(net, ln, b, wl.t0, wl.bin_width, wl.n_bins, policy, into=hab)
        perm = np.random.default_rng(seed).permutation(len(rec["ts"]))
        hp = o.discriminate_histogram(net, ln, {k: v[perm] for k, v in rec.items()}, wl.t0,
                                      wl.bin_width, wl.n_bins, policy)
        for k in ("count", "bytes", "stats"):
            assert np.array_equal(h[k], hab[k])
            assert np.array_equal(h[k], hp[k])


def check_count_wrap_and_wide_bytes(o):
    ts = np.array([5, 5], np.uint64)
    nb = np.array([0xFFFFFFFF, 0xFFFFFFFF], np.uint32)
    cls = np.array([1, 1], np.uint8)
    h = o.empty_hist(10)
    h["count"][0][5] = 0xFFFFFFFF
    o.histogram(ts, nb, cls, 0, 1, 10, oracle.EXCLUSIVE, into=h)
    assert int(h["count"][0][5]) == 1  # uint32 wraps modulo 2^32
    assert int(h["bytes"][0][5]) == 2 * 0xFFFFFFFF  # uint64 sum does not truncate


def check_sampled_bins(o, seed=9):
    wl = gen.scaled(gen.WORKLOADS["tiny"], 30_000)
    net, ln = gen.make_table(wl.table, wl.seed)
    rec = gen.make_records(wl.records, wl.seed, net, ln)
    nb = 2000
    w = 1800
    h = o.discriminate_histogram(net, ln, rec, 0, w, nb)
    keep = np.unique(np.random.default_rng(seed).integers(0, nb, 300)).astype(np.uint64)
    c, b = o.histogram_bins(net, ln, rec, 0, w, nb, keep)
    assert np.array_equal(c, h["count"][:, keep.astype(np.int64)])
    assert np.array_equal(b, h["bytes"][:, keep.astype(np.int64)])


def check_watch_filter(o, seed=13):
    """The watch filter against pins outside the oracle: a /0 list keeps every
    record; an empty list drops every record into stats[6]; a list of /32
    hosts keeps exactly the records numpy's isin selects."""
    wl = gen.scaled(gen.WORKLOADS["tiny"], 20_000)
    net, ln = gen.make_table(wl.table, wl.seed)
    rec = gen.make_records(wl.records, wl.seed, net, ln)
    full = o.discriminate_histogram(net, ln, rec, 0, 60_000, 60)
    every = o.discriminate_histogram_watch(net, ln, np.array([0], np.uint32), np.array([0], np.uint8), rec,
                                           0, 60_000, 60)
    for k in ("count", "bytes", "stats"):
        assert np.array_equal(every[k], full[k])
    none = o.discriminate_histogram_watch(net, ln, np.zeros(0, np.uint32), np.zeros(0, np.uint8), rec,
                                          0, 60_000, 60)
    assert int(none["stats"][6]) == len(rec["ts"]) and not none["count"].any() and not none["stats"][:6].any()
    rng = np.random.default_rng(seed)
    hosts = np.unique(np.concatenate([rng.choice(rec["src"], 150), rng.choice(rec["dst"], 150),
                                      rng.integers(0, 2 ** 32, 50, dtype=np.uint64).astype(np.uint32)]))
    watched = o.discriminate_histogram_watch(net, ln, hosts, np.full(len(hosts), 32, np.uint8), rec,
                                             0, 60_000, 60)
    keep = np.isin(rec["src"], hosts) | np.isin(rec["dst"], hosts)
    sub = o.discriminate_histogram(net, ln, {k: v[keep] for k, v in rec.items()}, 0, 60_000, 60)
    for k in ("count", "bytes"):
        assert np.array_equal(watched[k], sub[k])
    assert np.array_equal(watched["stats"][:6], sub["stats"][:6])
    assert int(watched["stats"][6]) == int((~keep).sum()) > 0 and keep.sum() > 0


CHECKS = [check_bitmask_golden, check_membership_golden, check_membership_ipaddress,
          check_membership_brute_force, check_class_bits, check_histogram_golden,
          check_histogram_numpy, check_brute_force_pipeline, check_invariants_generated,
          check_count_wrap_and_wide_bytes, check_sampled_bins, check_watch_filter]


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(orc, check):
    check(orc)


def test_minus_form_equals_equality():
    """Algorithm 1 compares with a subtraction: (SB - CB) mod 2^32 == 0 iff SB == CB."""
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2 ** 32, 200_000, dtype=np.uint64).astype(np.uint32)
    b = a.copy()
    flip = rng.random(len(a)) < 0.5
    b[flip] = rng.integers(0, 2 ** 32, int(flip.sum()), dtype=np.uint64).astype(np.uint32)
    with np.errstate(over="ignore"):
        assert np.array_equal((a - b) == 0, a == b)


# mutant id -> a short description (the mutations live in sinet_oracle.c)
MUTANTS = {1: "mask one bit short", 2: "/0 keeps all bits", 3: "CIDR host bits not masked",
           4: "src/dst class bits swapped", 5: "destination never tested",
           6: "window right edge included", 7: "records before t0 wrap",
           8: "policy read backwards", 9: "byte sums kept in 32 bits"}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda m: MUTANTS[m])
def test_planted_mistakes_are_caught(tmp_path, mutant):
    path = oracle.compile_variant(str(tmp_path / f"liboracle_m{mutant}.so"), mutant)
    o = oracle.Oracle(path)
    assert o.mutant() == mutant
    failed = []
    for check in CHECKS:
        try:
            check(o)
        except AssertionError:
            failed.append(check.__name__)
    assert failed, f"no pin caught planted mistake {mutant} ({MUTANTS[mutant]})"
