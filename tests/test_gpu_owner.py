"""Owner-computes strategy (SINET_STRAT_OWNER) against the oracle, bit-exact.

The strategy's own paths: records out of order by more than the tile's halo
(deferred strays), runs longer than one owner takes (overflow items), fully
unsorted input, every bin written by the owners (outputs that start as
garbage), the scalar store path (output arrays not 16-byte aligned),
accumulation, and the refusals. The general parity matrix runs the strategy
on every other case as well."""
from __future__ import annotations

import numpy as np
import pytest

import gen
from helpers import assert_hist_equal, run_fused, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2106_12863_gb300 as sinet  # noqa: E402

TABLE = gen.TableSpec(64, 16, 24)


@pytest.fixture(scope="module", autouse=True)
def lib():
    sinet.load()
    yield
    torch.cuda.synchronize()
    assert sinet.sinet_device_status() == 0


def _records(n, span_ms, jitter, seed, kind="diurnal"):
    net, ln = gen.make_table(TABLE, seed)
    spec = gen.RecordSpec(n, ts_kind=kind, t_lo=0, t_hi=span_ms, jitter=jitter)
    return net, ln, gen.make_records(spec, seed, net, ln)


@pytest.mark.parametrize("tile_bins", [16, 64, 0])
def test_jitter_beyond_halo(orc, tile_bins):
    # +-50 ms of disorder: beyond the halo of 16- and 64-slot tiles (4 and 16
    # bins), inside the default tile's; block boundaries defer strays in all
    net, ln, rec = _records(400_003, 200_000, 50, 21)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, 200_000)
    got = run_fused(sinet.PrefixTable(net, ln), to_dev(rec),
                    sinet.HistParams(0, 1, 200_000, strategy="owner", tile_bins=tile_bins))
    assert_hist_equal(got, ref, f"tile_bins={tile_bins}")


@pytest.mark.parametrize("tile_bins", [64, 0])
def test_dense_runs_overflow(orc, tile_bins):
    # 250 K records inside 8 ms (one range), the rest spread: runs far longer
    # than the 32,767 records an owner takes
    net, ln, rec = _records(300_001, 100_000, 0, 22)
    rng = np.random.default_rng(5)
    rec["ts"][:250_000] = rng.integers(5_000, 5_008, 250_000).astype(np.uint64)
    rec["bytes"][:1000] = 0xFFFFFFFF
    order = np.argsort(rec["ts"], kind="stable")
    rec = {k: v[order] for k, v in rec.items()}
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, 100_000)
    got = run_fused(sinet.PrefixTable(net, ln), to_dev(rec),
                    sinet.HistParams(0, 1, 100_000, strategy="owner", tile_bins=tile_bins,
                                     hints=sinet.HINT_TIME_SORTED))
    assert_hist_equal(got, ref, f"tile_bins={tile_bins}")


@pytest.mark.parametrize("width", [1, 7])
def test_unsorted_small_tiles(orc, width):
    # uniform (unsorted) timestamps: every range defers strays
    net, ln, rec = _records(200_003, 300_000, 0, 23, kind="uniform")
    t0, n_bins = 1234, 300_000 // width
    ref = orc.discriminate_histogram(net, ln, rec, t0, width, n_bins)
    got = run_fused(sinet.PrefixTable(net, ln), to_dev(rec),
                    sinet.HistParams(t0, width, n_bins, strategy="owner", tile_bins=16))
    assert_hist_equal(got, ref, f"width={width}")


@pytest.mark.parametrize("n_bins", [100_000, 100_001])
def test_every_bin_written(orc, n_bins):
    # outputs start as garbage and are not zeroed by the caller: the owners
    # store every bin and the counters start from zero. 100,001 bins leave
    # the second direction's arrays 4 bytes past a 16-byte boundary (the
    # scalar store path)
    net, ln, rec = _records(250_007, n_bins, 300, 24)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, n_bins)
    out = sinet.Histogram(n_bins, zero=False)
    out.count.fill_(-1)
    out.bytes.fill_(-1)
    out.stats.fill_(-1)
    d = to_dev(rec)
    sinet.discriminate_histogram(sinet.PrefixTable(net, ln), d["ts"], d["src"], d["dst"], d["bytes"],
                                 sinet.HistParams(0, 1, n_bins, strategy="owner"), out)
    torch.cuda.synchronize()
    assert_hist_equal(out.to_numpy(), ref, f"n_bins={n_bins}")


@pytest.mark.parametrize("n_bins", [100_000, 100_001])
def test_accumulate(orc, n_bins):
    net, ln, rec = _records(150_001, n_bins, 300, 25)
    t = sinet.PrefixTable(net, ln)
    d = to_dev(rec)
    out = sinet.Histogram(n_bins)
    p = sinet.HistParams(0, 1, n_bins, strategy="owner")
    sinet.discriminate_histogram(t, d["ts"], d["src"], d["dst"], d["bytes"], p, out)
    p.accumulate = True
    sinet.discriminate_histogram(t, d["ts"], d["src"], d["dst"], d["bytes"], p, out)
    torch.cuda.synchronize()
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, n_bins)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, n_bins, into=ref)
    assert_hist_equal(out.to_numpy(), ref, f"n_bins={n_bins}")


@pytest.mark.parametrize("strategy", ["owner", "auto"])
def test_sorted_hint(orc, strategy):
    net, ln, rec = _records(300_007, 3_600_000, 500, 26)
    ref = orc.discriminate_histogram(net, ln, rec, 0, 1, 3_600_000)
    got = run_fused(sinet.PrefixTable(net, ln), to_dev(rec),
                    sinet.HistParams(0, 1, 3_600_000, strategy=strategy, hints=sinet.HINT_TIME_SORTED))
    assert_hist_equal(got, ref, f"{strategy} + sorted hint")


@pytest.mark.parametrize("kw", [{"block_threads": 1024}, {"tile_bins": 8}])
def test_refused_shapes(kw):
    net, ln, rec = _records(1000, 10_000, 0, 27)
    d = to_dev(rec)
    out = sinet.Histogram(10_000)
    with pytest.raises(sinet.SinetError) as e:
        sinet.discriminate_histogram(sinet.PrefixTable(net, ln), d["ts"], d["src"], d["dst"], d["bytes"],
                                     sinet.HistParams(0, 1, 10_000, strategy="owner", **kw), out)
    assert e.value.status == 8
