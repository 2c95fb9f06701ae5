"""The owner-computes scheme's index arithmetic, restated on the host and
checked against a direct histogram (no GPU).

The scheme (SINET_STRAT_OWNER) rests on invariants of its partition and
store schedule rather than on atomics: the searched run boundaries form a
partition of the records for any input, the CTA blocks partition the
ranges, a circular tile of S slots never holds two bins in one slot, a
tile entry never counts past 16 bits, every bin is stored exactly once, and
every record is counted once. This test restates the steps (binary search,
prefix maximum, block split by records + bins, windows [b0 - H, b1 + H),
stores up to b1 - H, queued strays and overflow) with the kernel's
constants and asserts those invariants while building the histogram.
"""
from __future__ import annotations

import numpy as np
import pytest

CAP = 32767  # records an owner takes from one run


def _lower_bound(ts, key):
    lo, hi = 0, len(ts)
    while lo < hi:
        mid = lo + ((hi - lo) >> 1)
        if int(ts[mid]) < key:
            lo = mid + 1
        else:
            hi = mid
    return lo


def _owner(ts, by, dirs, t0, w, B, slots, G, halo=None, accumulate=False, init=None):
    n = len(ts)
    S = 16
    while S * 2 <= slots:
        S *= 2
    H = S // 4 if halo is None else halo
    T = S - 2 * H
    assert T % 4 == 0 and H % 4 == 0 and 2 * H <= T
    R = (B + T - 1) // T
    bounds = [0] + [_lower_bound(ts, t0 + k * T * w) for k in range(1, R)] + [n]
    bounds = list(np.maximum.accumulate(bounds))
    N = bounds[R] + B
    chi = lambda W: ((W + 1) * G - 1) // N  # noqa: E731
    part = [None] * (G + 1)
    for i in range(R + 1):
        W = bounds[i] + min(i * T, B)
        c_from = 0 if i == 0 else chi(bounds[i - 1] + min((i - 1) * T, B)) + 1
        for c in range(c_from, min(chi(W), G - 1) + 1):
            assert part[c] is None
            part[c] = i
    part[G] = R
    assert all(p is not None for p in part) and all(part[i] <= part[i + 1] for i in range(G))

    cnt = np.zeros((2, B), np.int64) if init is None else init[0].copy()
    byt = np.zeros((2, B), np.int64) if init is None else init[1].copy()
    stored = np.zeros(B, np.int64)
    counted = np.zeros(n, np.int64)
    oor = [0, 0]
    items = []

    def bin_of(i):
        rel = int(ts[i]) - t0
        return rel // w if 0 <= rel < B * w else None

    def count(i):
        counted[i] += 1
        if bin_of(i) is None:
            for d in range(2):
                oor[d] += dirs[i] >> d & 1

    for c in range(G):
        k0, k1 = part[c], part[c + 1]
        if k0 >= k1:
            continue
        lo, hi = k0 * T, min(k1 * T, B)
        tc = np.zeros((2, S), np.int64)
        tb = np.zeros((2, S), np.int64)
        tbin = np.full((2, S), -1, np.int64)
        for k in range(k0, k1):
            b0 = k * T
            b1 = min(b0 + T, B)
            wlo, whi = max(lo, b0 - H if b0 >= H else 0), min(hi, b1 + H)
            assert whi - wlo <= S
            ra, rb_run = bounds[k], bounds[k + 1]
            rb = min(rb_run, ra + CAP)
            stray = False
            for i in range(ra, rb):
                count(i)
                b = bin_of(i)
                if b is None or not dirs[i]:
                    continue
                if not wlo <= b < whi:
                    stray = True
                    continue
                s = b & (S - 1)
                for d in range(2):
                    if dirs[i] >> d & 1:
                        assert tc[d, s] == 0 or tbin[d, s] == b, "two bins in one slot"
                        tbin[d, s] = b
                        tc[d, s] += 1
                        tb[d, s] += int(by[i])
                        assert tc[d, s] < 1 << 16 and tb[d, s] < 1 << 48, "tile entry overflow"
            shi = b1 - H if k + 1 < k1 else hi
            assert wlo % 4 == 0 and wlo <= shi
            for b in range(wlo, shi):
                s = b & (S - 1)
                stored[b] += 1
                for d in range(2):
                    assert tc[d, s] == 0 or tbin[d, s] == b
                    cnt[d, b] = cnt[d, b] + tc[d, s] if accumulate else tc[d, s]
                    byt[d, b] = byt[d, b] + tb[d, s] if accumulate else tb[d, s]
                    tc[d, s] = tb[d, s] = 0
                    tbin[d, s] = -1
            if stray:
                items.append(("strays", ra, rb, wlo, whi))
            for x in range(rb, rb_run, CAP):
                items.append(("full", x, min(rb_run, x + CAP), b0, b1))
        assert not tc.any(), "tile not empty at the end of a block"
    assert len(items) <= R + n // CAP + 1
    for mode, x, y, wl, wh in items:  # the remainder kernel, after every owner stored its bins
        for i in range(x, y):
            if mode == "full":
                count(i)
            b = bin_of(i)
            if b is None or (mode == "strays" and wl <= b < wh):
                continue
            for d in range(2):
                if dirs[i] >> d & 1:
                    cnt[d, b] += 1
                    byt[d, b] += int(by[i])
    assert (counted == 1).all(), "a record counted other than once"
    if not accumulate:
        assert (stored == 1).all(), "a bin stored other than once"
    return cnt, byt, oor


def _direct(ts, by, dirs, t0, w, B):
    cnt = np.zeros((2, B), np.int64)
    byt = np.zeros((2, B), np.int64)
    oor = [0, 0]
    for i in range(len(ts)):
        rel = int(ts[i]) - t0
        for d in range(2):
            if dirs[i] >> d & 1:
                if 0 <= rel < B * w:
                    cnt[d, rel // w] += 1
                    byt[d, rel // w] += int(by[i])
                else:
                    oor[d] += 1
    return cnt, byt, oor


def _inputs(kind, seed, n=4000, span=4000):
    rng = np.random.default_rng(seed)
    if kind == "jitter":
        ts = np.clip(np.sort(rng.integers(0, span, n)) + rng.integers(-40, 41, n), 0, None)
    elif kind == "dense":
        ts = np.sort(np.concatenate([rng.integers(300, 303, 3 * CAP // 2), rng.integers(0, span, n)]))
    else:
        ts = rng.integers(0, span + 500, n)
    ts = ts.astype(np.uint64)
    m = len(ts)
    return ts, rng.integers(0, 2 ** 32, m, dtype=np.uint64), rng.integers(0, 4, m)


@pytest.mark.parametrize("kind,slots,G,halo", [
    ("jitter", 16, 1, None), ("jitter", 64, 5, None), ("jitter", 64, 5, 8), ("jitter", 4096, 304, None),
    ("dense", 64, 3, None), ("dense", 4096, 304, None),
    ("unsorted", 16, 7, None), ("unsorted", 256, 2, 32),
])
def test_scheme_equals_direct_histogram(kind, slots, G, halo):
    ts, by, dirs = _inputs(kind, 7)
    t0, w, B = 100, 1, 3900
    got = _owner(ts, by, dirs, t0, w, B, slots, G, halo)
    want = _direct(ts, by, dirs, t0, w, B)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]) and got[2] == want[2]


def test_wide_bins_tiny_inputs_and_more_ctas_than_ranges():
    ts, by, dirs = _inputs("jitter", 8, n=300, span=3000)
    for t0, w, B, slots, G in ((0, 1000, 3, 64, 9), (0, 1, 61, 4096, 304), (0, 1, 3000, 16, 1000)):
        got = _owner(ts, by, dirs, t0, w, B, slots, G)
        want = _direct(ts, by, dirs, t0, w, B)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]) and got[2] == want[2]


def test_accumulate_adds_onto_the_arrays():
    ts, by, dirs = _inputs("jitter", 9)
    first = _owner(ts, by, dirs, 0, 1, 4000, 64, 7)
    again = _owner(ts, by, dirs, 0, 1, 4000, 64, 7, accumulate=True, init=first[:2])
    want = _direct(ts, by, dirs, 0, 1, 4000)
    assert np.array_equal(again[0], 2 * want[0]) and np.array_equal(again[1], 2 * want[1])
