"""The allocation-free entry point, checked against the allocating one.

``sinet_discriminate_histogram_noalloc`` serves callers that cannot allocate
device memory on the call path: it runs the plain sort + reduce-by-key path
with its scratch in a fixed device array built into the library. Here it is
called twice in a row through the C ABI (the second time on different, smaller
input, so the array still holds the first call's contents) and each result is
compared with ``sinet_discriminate_histogram`` on the same input. The
tolerance is zero, as for every other parity test: the arithmetic is integer.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

import gen

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
    return w, net, ln, d


def _run(fn, table, d, params):
    out = sinet.Histogram(params.n_bins)
    fn(table.handle, d["ts"], d["src"], d["dst"], d["bytes"], d["ts"].numel(), params.c(), out.c())
    torch.cuda.synchronize()
    return out.to_numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_2106_12863_gb300 import _build

    _build.build()
    sinet.load()
    cases = [("tiny", 1_000_003, 0, sinet.EXCLUSIVE), ("day", 600_001, 5, sinet.INCLUSIVE)]
    for key, n, shift, policy in cases:
        w, net, ln, d = _inputs(key, n, shift)
        table = sinet.PrefixTable(net, ln)
        params = sinet.HistParams(w.t0, w.bin_width, w.n_bins, policy=policy)
        want = _run(sinet.sinet_discriminate_histogram, table, d, params)
        got = _run(sinet.sinet_discriminate_histogram_noalloc, table, d, params)
        for k in ("count", "bytes", "stats"):
            assert np.array_equal(got[k], want[k]), (key, k)
        assert int(got["stats"][:4].sum()) == n
        assert int(got["stats"][7]) == 0  # no device-side failure latched
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
