"""The allocation-free entry point, against the oracle and the allocating one.

``sinet_discriminate_histogram_noalloc`` serves callers that cannot allocate
device memory on the call path (a host application whose own memory manager
owns every device allocation, or a latency-bound loop where an allocator call
could synchronise the device or fail under fragmentation): it runs the plain
sort + reduce-by-key path with its scratch in a fixed device array built into
the library. Here it is called through the C ABI twice in a row (the second
time on different, smaller input, so the array still holds the first call's
contents); each result must equal the CPU oracle and
``sinet_discriminate_histogram`` on the same input, element by element (the
tolerance is zero, as for every other parity test: the arithmetic is
integer). An accumulating call must add onto the previous result and clear a
stale status left in stats[7]. This file is collected last so that a run
stopping at the first failure has already run every other test; it builds
nothing itself (``__graft_entry__.build()`` does).
"""
from __future__ import annotations

import numpy as np
import pytest

import gen
from helpers import assert_hist_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2106_12863_gb300 as sinet  # noqa: E402


def _inputs(key, n, seed_shift):
    w = gen.scaled(gen.WORKLOADS[key], n)
    net, ln = gen.make_table(w.table, w.seed + seed_shift)
    rec = gen.make_records(w.records, w.seed + seed_shift, net, ln)
    d = {"ts": torch.from_numpy(rec["ts"].view(np.int64)).cuda(),
         "src": torch.from_numpy(rec["src"].view(np.int32)).cuda(),
         "dst": torch.from_numpy(rec["dst"].view(np.int32)).cuda(),
         "bytes": torch.from_numpy(rec["bytes"].view(np.int32)).cuda()}
    return w, net, ln, rec, d


def _run(fn, table, d, params, out=None):
    out = out or sinet.Histogram(params.n_bins)
    fn(table.handle, d["ts"], d["src"], d["dst"], d["bytes"], d["ts"].numel(), params.c(), out.c())
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_oracle_and_allocating_entry_point_twice(orc):
    sinet.load()
    cases = [("tiny", 1_000_003, 0, sinet.EXCLUSIVE), ("day", 600_001, 5, sinet.INCLUSIVE)]
    for key, n, shift, policy in cases:
        w, net, ln, rec, d = _inputs(key, n, shift)
        table = sinet.PrefixTable(net, ln)
        params = sinet.HistParams(w.t0, w.bin_width, w.n_bins, policy=policy)
        ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins, policy)
        want = _run(sinet.sinet_discriminate_histogram, table, d, params).to_numpy()
        got = _run(sinet.sinet_discriminate_histogram_noalloc, table, d, params).to_numpy()
        assert_hist_equal(got, ref, f"noalloc {key} vs oracle")
        assert_hist_equal(got, want, f"noalloc {key} vs allocating")
        assert int(got["stats"][:4].sum()) == n
        assert int(got["stats"][7]) == 0  # no device-side failure latched
        table.close()


def test_noalloc_accumulates_and_clears_a_stale_status(orc):
    sinet.load()
    w, net, ln, rec, d = _inputs("tiny", 300_007, 9)
    table = sinet.PrefixTable(net, ln)
    params = sinet.HistParams(w.t0, w.bin_width, w.n_bins)
    out = _run(sinet.sinet_discriminate_histogram_noalloc, table, d, params)
    out.stats[7] = 0xDEAD  # a status a previous call might have left behind
    params.accumulate = True
    got = _run(sinet.sinet_discriminate_histogram_noalloc, table, d, params, out).to_numpy()
    ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    ref = orc.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins, into=ref)
    assert int(got["stats"][7]) & 0xFFFFFFFF == 0
    got["stats"][7] = 0
    assert_hist_equal(got, ref, "noalloc accumulate")
    table.close()


def test_noalloc_rejects_inputs_beyond_its_array():
    sinet.load()
    w = gen.WORKLOADS["tiny"]
    net, ln = gen.make_table(w.table, w.seed)
    table = sinet.PrefixTable(net, ln)
    n = 4_000_000  # needs more than the fixed 32 MiB of scratch
    big = torch.zeros(n, dtype=torch.int64, device="cuda")
    small = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = sinet.Histogram(16)
    with pytest.raises(sinet.SinetError) as e:
        sinet.sinet_discriminate_histogram_noalloc(table.handle, big, small, small, small, n,
                                                   sinet.HistParams(0, 1, 16).c(), out.c())
    assert e.value.status == 4  # SINET_ERR_BUDGET, nothing launched
    table.close()
