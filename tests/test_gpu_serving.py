"""GPU tests of the continuous-batching serving loop: every tenant's resident
histogram equals the oracle summed over that tenant's requests, bit-exact,
whether the requests are served one at a time or mixed into shared launches;
admission by budget and slots; host-side timeouts."""
from __future__ import annotations

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2106_12863_gb300 as sinet  # noqa: E402

# tenant windows: the whole day at several widths (tile, combining, plain atomics)
WIDTHS = [(60_000, "auto"), (100, "global_atomic"), (1000, "atomic_noagg"), (10, "auto")]


@pytest.fixture(scope="module", autouse=True)
def lib():
    sinet.load()
    yield
    torch.cuda.synchronize()
    assert sinet.sinet_device_status() == 0


@pytest.fixture(scope="module")
def stream_():
    specs, reqs = gen.serving_plan(n_tenants=len(WIDTHS), n_requests=36, median=30_000, cap=400_000,
                                   p_lo=500, p_hi=4000)
    tables = [gen.make_table(s, 900 + i) for i, s in enumerate(specs)]
    data = []
    for r in reqs:
        net, ln = tables[r.tenant]
        rec = gen.make_records(r.records, r.seed, net, ln)
        data.append((r.tenant, rec))
    # one empty request and one with records outside its tenant's window
    data.append((1, {k: v[:0] for k, v in data[0][1].items()}))
    late = dict(data[1][1])
    late["ts"] = late["ts"] + np.uint64(gen.DAY_MS)
    data.append((data[1][0], late))
    return tables, data


def _params(i):
    w, strat = WIDTHS[i]
    return sinet.HistParams(0, w, -(-gen.DAY_MS // w), strategy=strat, accumulate=True)


def _want(orc, tables, data):
    out = []
    for i in range(len(WIDTHS)):
        p = _params(i)
        h = orc.empty_hist(p.n_bins)
        net, ln = tables[i]
        for t, rec in data:
            if t == i:
                orc.discriminate_histogram(net, ln, rec, p.t0_ms, p.bin_width_ms, p.n_bins, into=h)
        out.append(h)
    return out


def _server(tables, budget, per_launch):
    ptabs = [sinet.PrefixTable(*t) for t in tables]
    s = sinet.Server([(ptabs[i], _params(i)) for i in range(len(WIDTHS))], budget_bytes=budget,
                     max_requests_per_launch=per_launch)
    return s, ptabs


def _check(server, want):
    for i, w in enumerate(want):
        got = server.export(i)
        for k in ("stats", "count", "bytes"):
            assert np.array_equal(got[k], w[k]), f"tenant {i} {k}"


def test_serving_alone_equals_mix_equals_oracle(orc, stream_):
    tables, data = stream_
    want = _want(orc, tables, data)
    # mixed: everything submitted at once; a small arena and few slots per
    # launch force staged admission and many shared launches
    mix, _t1 = _server(tables, budget=24 << 20, per_launch=5)
    pinned = []
    for t, rec in data:
        bufs = [torch.from_numpy(rec[k].view(np.int64 if k == "ts" else np.int32)).pin_memory()
                for k in ("ts", "src", "dst", "bytes")]
        pinned.append((t, bufs))
    tickets = [mix.submit(t, *b) for t, b in pinned]
    infos = [mix.wait(k) for k in tickets]
    mix.drain()
    st = mix.stats()
    assert st["requests_done"] == len(data)
    assert st["records_done"] == sum(len(r["ts"]) for _, r in data)
    assert st["launches"] < len(data)  # requests shared launches
    assert max(i["launch"] for i in infos) == st["launches"]
    assert st["p50_latency_ns"] <= st["p99_latency_ns"] <= st["max_latency_ns"]
    _check(mix, want)
    mix.close()
    # alone: one request in flight at a time, pageable numpy buffers
    alone, _t2 = _server(tables, budget=64 << 20, per_launch=64)
    for t, rec in data:
        k = alone.submit(t, rec["ts"], rec["src"], rec["dst"], rec["bytes"])
        info = alone.wait(k)
        assert info["n"] == len(rec["ts"])
    assert alone.stats()["launches"] == len(data)
    _check(alone, want)
    alone.close()


def test_serving_admission_and_timeouts(stream_):
    tables, data = stream_
    s, _t = _server(tables, budget=1 << 20, per_launch=4)
    big = 60_000  # 1.2 MB of records: larger than the whole 1 MiB arena
    z64, z32 = np.zeros(big, np.uint64), np.zeros(big, np.uint32)
    with pytest.raises(sinet.SinetError) as ei:
        s.submit(0, z64, z32, z32, z32)
    assert ei.value.status == 4  # SINET_ERR_BUDGET
    with pytest.raises(sinet.SinetError) as ei:
        s.submit(len(WIDTHS), z64[:1], z32[:1], z32[:1], z32[:1])
    assert ei.value.status == 1
    with pytest.raises(sinet.SinetError) as ei:
        s.wait(12345)
    assert ei.value.status == 1
    # many requests that together exceed the arena: admitted as space frees
    rec = data[0][1]
    n = min(len(rec["ts"]), 20_000)
    ks = [s.submit(data[0][0], rec["ts"][:n], rec["src"][:n], rec["dst"][:n], rec["bytes"][:n])
          for _ in range(12)]
    for k in ks:
        s.wait(k)
    s.drain()
    s.close()
    # outstanding-request limit
    ptabs = [sinet.PrefixTable(*t) for t in tables]
    s2 = sinet.Server([(ptabs[i], _params(i)) for i in range(len(WIDTHS))], budget_bytes=64 << 20,
                      max_requests_per_launch=4, max_queued=2)
    n = len(rec["ts"])
    k1 = s2.submit(0, rec["ts"], rec["src"], rec["dst"], rec["bytes"])
    k2 = s2.submit(0, rec["ts"], rec["src"], rec["dst"], rec["bytes"])
    try:
        s2.submit(0, rec["ts"], rec["src"], rec["dst"], rec["bytes"])
        third = True  # the first two may already be done
    except sinet.SinetError as e:
        assert e.status == 4
        third = False
    s2.wait(k1)
    s2.wait(k2)
    s2.drain()
    if not third:
        assert s2.stats()["requests_done"] == 2
    s2.close()
    assert n > 0


def test_serving_checkpoint_round_trip(orc, stream_):
    """Export a tenant, import it into a fresh server, keep serving there: the
    result equals serving everything on one server (and the oracle)."""
    tables, data = stream_
    want = _want(orc, tables, data)
    half = len(data) // 2
    a, _ta = _server(tables, budget=64 << 20, per_launch=8)
    for t, rec in data[:half]:
        a.wait(a.submit(t, rec["ts"], rec["src"], rec["dst"], rec["bytes"]))
    a.drain()
    snap = [a.export(i) for i in range(len(WIDTHS))]
    a.close()
    b, _tb = _server(tables, budget=64 << 20, per_launch=8)
    for i, h in enumerate(snap):
        b.import_(i, h)
        back = b.export(i)
        for k in ("stats", "count", "bytes"):
            assert np.array_equal(back[k], h[k]), f"tenant {i} {k} round trip"
    ks = [b.submit(t, rec["ts"], rec["src"], rec["dst"], rec["bytes"]) for t, rec in data[half:]]
    for k in ks:
        b.wait(k)
    b.drain()
    _check(b, want)
    b.close()
