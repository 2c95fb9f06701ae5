"""GPU parity of the histogram post-processing: roll-up into coarser bins
(against the oracle run directly at the coarser width, and against a numpy
reshape-sum of the oracle's fine histogram) and sparse compaction (against
numpy's non-zero selection), bit-exact."""
from __future__ import annotations

import numpy as np
import pytest

import gen
from helpers import run_fused, to_dev

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


@pytest.fixture(scope="module")
def tiny():
    w = gen.scaled(gen.WORKLOADS["tiny"], 300_007)
    net, ln = gen.make_table(w.table, w.seed)
    rec = gen.make_records(w.records, w.seed, net, ln)
    return w, net, ln, rec


def _dev_hist(h):
    out = sinet.Histogram(h["count"].shape[1])
    out.count.copy_(torch.from_numpy(h["count"].view(np.int32)))
    out.bytes.copy_(torch.from_numpy(h["bytes"].view(np.int64)))
    out.stats.copy_(torch.from_numpy(h["stats"].view(np.int64)))
    return out


def _reshape_sum(h, factor):
    nb = h["count"].shape[1]
    n_out = -(-nb // factor)
    pad = n_out * factor - nb
    c = np.pad(h["count"].astype(np.uint64), ((0, 0), (0, pad))).reshape(2, n_out, factor).sum(axis=2)
    with np.errstate(over="ignore"):
        b = np.pad(h["bytes"], ((0, 0), (0, pad))).reshape(2, n_out, factor).sum(axis=2, dtype=np.uint64)
    return (c & 0xFFFFFFFF).astype(np.uint32), b


@pytest.mark.parametrize("factor", [1, 7, 1000, 60_000, 3_600_000, 10_000_000])
def test_rollup_equals_direct_coarse_histogram(orc, tiny, factor):
    w, net, ln, rec = tiny
    fine = run_fused(sinet.PrefixTable(net, ln), to_dev(rec), sinet.HistParams(w.t0, 1, w.n_bins))
    got = sinet.rollup(_dev_hist(fine), factor).to_numpy()
    c, b = _reshape_sum(fine, factor)
    assert np.array_equal(got["count"], c) and np.array_equal(got["bytes"], b)
    assert np.array_equal(got["stats"], fine["stats"])
    # the oracle at the coarse width (the window becomes whole coarse bins)
    n_out = -(-w.n_bins // factor)
    want = orc.discriminate_histogram(net, ln, rec, w.t0, factor, n_out)
    assert np.array_equal(got["count"], want["count"])
    assert np.array_equal(got["bytes"], want["bytes"])


def test_rollup_accumulates(orc, tiny):
    w, net, ln, rec = tiny
    fine = orc.discriminate_histogram(net, ln, rec, w.t0, 1, w.n_bins)
    out = sinet.rollup(_dev_hist(fine), 997)
    sinet.rollup(_dev_hist(fine), 997, out=out, accumulate=True)
    c, b = _reshape_sum(fine, 997)
    got = out.to_numpy()
    with np.errstate(over="ignore"):
        assert np.array_equal(got["count"], c * np.uint32(2))
        assert np.array_equal(got["bytes"], b * np.uint64(2))


@pytest.mark.parametrize("n_bins", [1, 4095, 4096, 4097, 3_600_000])
def test_sparse_equals_nonzero(orc, tiny, n_bins):
    w, net, ln, rec = tiny
    h = orc.discriminate_histogram(net, ln, rec, w.t0, max(1, w.n_bins // n_bins), n_bins)
    got = sinet.sparse(_dev_hist(h))
    keep = np.flatnonzero((h["count"][0] | h["count"][1]) != 0)
    assert got["n"] == len(keep)
    assert np.array_equal(got["bin"].cpu().numpy().view(np.uint32), keep.astype(np.uint32))
    assert np.array_equal(got["count"].cpu().numpy().view(np.uint32), h["count"][:, keep])
    assert np.array_equal(got["bytes"].cpu().numpy().view(np.uint64), h["bytes"][:, keep])


def test_sparse_capacity_and_empty(orc, tiny):
    w, net, ln, rec = tiny
    h = orc.discriminate_histogram(net, ln, rec, w.t0, 1, w.n_bins)
    keep = np.flatnonzero((h["count"][0] | h["count"][1]) != 0)
    got = sinet.sparse(_dev_hist(h), cap=1000)
    assert got["n"] == len(keep) and len(got["bin"]) == 1000
    assert np.array_equal(got["bin"].cpu().numpy().view(np.uint32), keep[:1000].astype(np.uint32))
    empty = sinet.Histogram(5000)
    assert sinet.sparse(empty)["n"] == 0
