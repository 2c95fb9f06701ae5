"""The device division by the bin width (an invariant-divisor multiply after
Granlund & Montgomery) against the CPU's integer division, through
``sinet_bin``: numerators at and around the window's edges, widths that are
powers of two, one off a power of two, primes and near 2^63, and windows whose
end lies close to 2^64."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2106_12863_gb300 as sinet  # noqa: E402

NONE = 0xFFFFFFFF


def _widths():
    ws = {1, 2, 3, 7, 10, 1000, 60_000, 3_600_000, 999_983, 86_400_000}
    for k in range(1, 64):
        for d in (-1, 0, 1):
            v = (1 << k) + d
            if 1 <= v < (1 << 64):
                ws.add(v)
    ws |= {(1 << 63) - 25, (1 << 63) + 29, (1 << 64) - 59}  # primes around 2^63 and below 2^64
    return sorted(ws)


def _case(t0, w, n_bins, rng):
    span = n_bins * w
    rel = [0, 1, w - 1, w, w + 1, span - w, span - w - 1, span - 1, span, span + 1]
    hi_, lo_ = rng.integers(0, 1 << 32, 200), rng.integers(0, 1 << 32, 200)
    rel += [(int(a) << 32 | int(b)) % span for a, b in zip(hi_, lo_)]
    rel += [(int(q) * w + r) for q in rng.integers(0, n_bins, 50) for r in (0, w - 1)]
    rel = [r for r in rel if 0 <= r < (1 << 64) - t0] + [-1, -w]  # and before t0 (wraps)
    vals = [(t0 + r) % (1 << 64) for r in rel]
    # built from 32-bit halves: Python ints of 2^63 and above do not convert directly
    ts = (np.array([v >> 32 for v in vals], np.uint64) << np.uint64(32)) | np.array(
        [v & 0xFFFFFFFF for v in vals], np.uint64)
    want = np.array([(v - t0) // w if t0 <= v < t0 + span else NONE for v in vals], np.uint32)
    return ts, want


@pytest.mark.parametrize("t0_kind", ["zero", "mid", "near_top"])
def test_divider_against_integer_division(t0_kind):
    sinet.load()
    rng = np.random.default_rng(7)
    ts_all, want_all = [], []
    for w in _widths():
        n_bins = int(min((1 << 31) - 1, max(1, ((1 << 64) - 1) // w // 2)))
        n_bins = int(min(n_bins, rng.integers(1, 1 << 31)))
        span = n_bins * w
        t0 = {"zero": 0, "mid": (1 << 62) + 12345, "near_top": (1 << 64) - 1 - span}[t0_kind]
        if t0 + span >= (1 << 64):
            continue
        ts, want = _case(t0, w, n_bins, rng)
        d = torch.from_numpy(ts.view(np.int64)).cuda()
        got = sinet.bin_index(d, t0, w, n_bins)
        torch.cuda.synchronize()
        g = got.cpu().numpy().view(np.uint32)
        bad = np.nonzero(g != want)[0]
        assert len(bad) == 0, f"w={w} t0={t0} n_bins={n_bins}: ts={ts[bad[0]]} got {g[bad[0]]} want {want[bad[0]]}"
        ts_all.append(ts)
        want_all.append(want)
    assert sum(len(x) for x in ts_all) > 10_000


def test_bin_refuses_bad_parameters():
    sinet.load()
    d = torch.zeros(4, dtype=torch.int64, device="cuda")
    o = torch.empty(4, dtype=torch.int32, device="cuda")
    for t0, w, nb in ((0, 0, 10), (0, 1, 0), (0, 1, 1 << 31), ((1 << 64) - 5, 1, 10)):
        with pytest.raises(sinet.SinetError) as e:
            sinet.sinet_bin(d, 4, t0, w, nb, o)
        assert e.value.status == 1
