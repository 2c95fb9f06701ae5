"""Shared helpers for the GPU tests: moving records to the device, running the
library through the C ABI, and comparing with the oracle element by element."""
from __future__ import annotations

import numpy as np


def to_dev(rec: dict, device="cuda", offsets=None):
    """Copy numpy SoA records to CUDA tensors. ``offsets`` (per field, in
    elements) places each stream at a deliberately unaligned start."""
    import torch

    out = {}
    for k, v in rec.items():
        if k not in ("ts", "src", "dst", "bytes", "cls"):
            continue
        if v.dtype == np.uint64:
            a = v.view(np.int64)
        elif v.dtype == np.uint32:
            a = v.view(np.int32)
        else:
            a = v
        off = (offsets or {}).get(k, 0)
        t = torch.from_numpy(np.ascontiguousarray(a))
        if off:
            buf = torch.zeros(len(a) + off, dtype=t.dtype, device=device)
            buf[off:] = t.to(device)
            out[k] = buf[off:]
        else:
            out[k] = t.to(device)
    return out


def assert_hist_equal(got: dict, ref: dict, what=""):
    for k in ("stats", "count", "bytes"):
        g, r = got[k], ref[k]
        if not np.array_equal(g, r):
            bad = np.argwhere(g != r)
            i = tuple(bad[0])
            raise AssertionError(f"{what}: {k} differs at {len(bad)} places; first {i}: "
                                 f"got {g[i]} want {r[i]}")


def run_fused(table, dev: dict, params, device="cuda"):
    import paper_2106_12863_gb300 as sinet
    import torch

    out = sinet.Histogram(params.n_bins, device)
    sinet.discriminate_histogram(table, dev["ts"], dev["src"], dev["dst"], dev["bytes"], params, out)
    torch.cuda.synchronize()
    return out.to_numpy()
