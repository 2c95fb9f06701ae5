"""Thin ctypes binding over ``libsinet.so`` (the C ABI declared in include/sinet.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library. Functions named ``sinet_*`` mirror the C entry points one to one;
``PrefixTable``, ``HistParams``, ``Histogram`` and the lower-case helpers are
conveniences over them. Device buffers are torch CUDA tensors (uint64 data as
int64, uint32 as int32, reinterpreted bit for bit). The library must be built
(``__graft_entry__.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsinet.so")

OK = 0
STATUS = {0: "SINET_OK", 1: "SINET_ERR_INVALID_ARG", 2: "SINET_ERR_CUDA", 3: "SINET_ERR_OOM",
          4: "SINET_ERR_BUDGET", 5: "SINET_ERR_TIMEOUT", 6: "SINET_ERR_TABLE_TOO_LARGE",
          7: "SINET_ERR_DEVICE_CHECK", 8: "SINET_ERR_UNSUPPORTED"}

STRAT_AUTO, STRAT_GLOBAL_ATOMIC, STRAT_PRIV_TILE, STRAT_SORT_REDUCE, STRAT_SMEM_FULL, \
    STRAT_ATOMIC_NOAGG, STRAT_ATOMIC_CELL, STRAT_OWNER, STRAT_PARTITION = range(9)
STRATEGIES = {"auto": STRAT_AUTO, "global_atomic": STRAT_GLOBAL_ATOMIC,
              "priv_tile": STRAT_PRIV_TILE, "sort_reduce": STRAT_SORT_REDUCE,
              "smem_full": STRAT_SMEM_FULL, "atomic_noagg": STRAT_ATOMIC_NOAGG,
              "atomic_cell": STRAT_ATOMIC_CELL, "owner": STRAT_OWNER,
              "partition": STRAT_PARTITION}
LOOKUP_AUTO, LOOKUP_INTERVAL, LOOKUP_PML = range(3)
LOOKUPS = {"auto": LOOKUP_AUTO, "interval": LOOKUP_INTERVAL, "pml": LOOKUP_PML}
HINT_TIME_SORTED = 1
HINT_TUNE = 2

DIR_OUT, DIR_IN = 1, 2
EXCLUSIVE = (0, DIR_OUT, DIR_IN, 0)
PAPER_ALG1 = (DIR_IN, DIR_OUT, DIR_IN, DIR_OUT)
INCLUSIVE = (0, DIR_OUT, DIR_IN, DIR_OUT | DIR_IN)


class SinetError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class HistParamsC(ctypes.Structure):
    _fields_ = [("t0_ms", ctypes.c_uint64), ("bin_width_ms", ctypes.c_uint64),
                ("n_bins", ctypes.c_uint64), ("policy", ctypes.c_uint8 * 4),
                ("accumulate", ctypes.c_int32), ("strategy", ctypes.c_int32),
                ("lookup", ctypes.c_int32), ("hints", ctypes.c_uint32),
                ("tile_bins", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("watch", ctypes.c_void_p)]


class HistOutC(ctypes.Structure):
    _fields_ = [("count", ctypes.c_void_p * 2), ("bytes", ctypes.c_void_p * 2),
                ("stats", ctypes.c_void_p)]


class BatchSliceC(ctypes.Structure):
    _fields_ = [("ts", ctypes.c_void_p), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("bytes", ctypes.c_void_p), ("n", ctypes.c_uint64), ("table", ctypes.c_void_p),
                ("params", HistParamsC), ("out", HistOutC), ("ready", ctypes.c_void_p),
                ("ready_value", ctypes.c_uint32)]


BATCH_AUTOTUNE = 1


class TenantC(ctypes.Structure):
    _fields_ = [("table", ctypes.c_void_p), ("params", HistParamsC)]


class ServerConfigC(ctypes.Structure):
    _fields_ = [("inflight_budget_bytes", ctypes.c_uint64), ("max_requests_per_launch", ctypes.c_uint32),
                ("max_queued", ctypes.c_uint32)]


class RequestInfoC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("launch", ctypes.c_uint64), ("latency_ns", ctypes.c_uint64)]


class ServerCountersC(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_uint64), ("records_done", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("p50_latency_ns", ctypes.c_uint64),
                ("p99_latency_ns", ctypes.c_uint64), ("max_latency_ns", ctypes.c_uint64),
                ("busy_ns", ctypes.c_uint64)]

_lib = None
_P = ctypes.c_void_p


def load():
    """Load libsinet.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
    sig = {
        "sinet_version": (u32, []),
        "sinet_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "sinet_last_cuda_error": (ctypes.c_int, []),
        "sinet_parse_cidr": (ctypes.c_int, [ctypes.c_char_p, _P, _P]),
        "sinet_compile_prefix_table": (ctypes.c_int, [_P, _P, u32, u32, _P, _P, _P, _P, _P, _P]),
        "sinet_prefix_table_image": (ctypes.c_int, [_P, _P, u32, _P, ctypes.c_size_t, _P, _P]),
        "sinet_build_prefix_table": (ctypes.c_int, [_P, _P, u32, _P, _P]),
        "sinet_destroy_prefix_table": (ctypes.c_int, [_P]),
        "sinet_discriminate": (ctypes.c_int, [_P, _P, _P, u64, _P, _P, i32, _P]),
        "sinet_bin": (ctypes.c_int, [_P, u64, u64, u64, u64, _P, _P]),
        "sinet_histogram": (ctypes.c_int, [_P, _P, _P, u64, ctypes.POINTER(HistParamsC),
                                           ctypes.POINTER(HistOutC), _P]),
        "sinet_discriminate_histogram": (ctypes.c_int, [_P, _P, _P, _P, _P, u64,
                                                        ctypes.POINTER(HistParamsC),
                                                        ctypes.POINTER(HistOutC), _P]),
        "sinet_discriminate_histogram_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, u64,
                                                                ctypes.POINTER(HistParamsC),
                                                                ctypes.POINTER(HistOutC), _P]),
        "sinet_device_status": (ctypes.c_int, [_P, _P]),
        "sinet_auto_strategy": (ctypes.c_int, [_P, u64, ctypes.POINTER(HistParamsC), _P]),
        "sinet_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchSliceC), u32, u32, _P, _P]),
        "sinet_batch_run": (ctypes.c_int, [_P, _P]),
        "sinet_batch_strategy": (ctypes.c_int, [_P, u32, _P]),
        "sinet_batch_set_wait": (ctypes.c_int, [_P, u64]),
        "sinet_batch_info": (ctypes.c_int, [_P, _P, _P]),
        "sinet_batch_destroy": (ctypes.c_int, [_P]),
        "sinet_histogram_rollup": (ctypes.c_int, [ctypes.POINTER(HistOutC), u64, u64, ctypes.c_int,
                                                  ctypes.POINTER(HistOutC), _P]),
        "sinet_histogram_sparse": (ctypes.c_int, [ctypes.POINTER(HistOutC), u64, _P, _P, _P, _P, _P, u64, _P, _P]),
        "sinet_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfigC), ctypes.POINTER(TenantC), u32, _P]),
        "sinet_server_submit": (ctypes.c_int, [_P, u32, _P, _P, _P, _P, u64, _P]),
        "sinet_server_wait": (ctypes.c_int, [_P, u64, u32, _P]),
        "sinet_server_drain": (ctypes.c_int, [_P, u32]),
        "sinet_server_tenant_output": (ctypes.c_int, [_P, u32, ctypes.POINTER(HistOutC)]),
        "sinet_server_export": (ctypes.c_int, [_P, u32, _P, _P, _P]),
        "sinet_server_import": (ctypes.c_int, [_P, u32, _P, _P, _P]),
        "sinet_server_stats": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ServerCountersC)]),
        "sinet_server_destroy": (ctypes.c_int, [_P]),
        "sinet_default_params": (None, [ctypes.POINTER(HistParamsC), u64, u64, u64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != OK:
        raise SinetError(rc, where)


def _dptr(t) -> int | None:
    """Device pointer of a CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> int | None:
    import torch

    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# C entry points, same names


def sinet_version() -> int:
    return int(load().sinet_version())


def sinet_parse_cidr(text: str):
    net, ln = ctypes.c_uint32(), ctypes.c_uint8()
    _check(load().sinet_parse_cidr(text.encode(), ctypes.byref(net), ctypes.byref(ln)),
           f"sinet_parse_cidr({text!r})")
    return int(net.value), int(ln.value)


def sinet_compile_prefix_table(net, ln, index_bits: int = 0) -> dict:
    net = np.ascontiguousarray(net, np.uint32)
    ln = np.ascontiguousarray(ln, np.uint8)
    n = len(net)
    counts = np.zeros(4, np.uint32)
    off = np.zeros(34, np.uint32)
    # first pass: sizes
    _check(load().sinet_compile_prefix_table(net.ctypes.data, ln.ctypes.data, n, index_bits, None,
                                             off.ctypes.data, None, None, None, counts.ctypes.data),
           "sinet_compile_prefix_table")
    nets = np.zeros(max(n, 1), np.uint32)
    lo = np.zeros(max(n, 1), np.uint32)
    hi = np.zeros(max(n, 1), np.uint32)
    index = np.zeros((1 << int(counts[2])) + 1, np.uint32)
    _check(load().sinet_compile_prefix_table(net.ctypes.data, ln.ctypes.data, n, index_bits,
                                             nets.ctypes.data, off.ctypes.data, lo.ctypes.data,
                                             hi.ctypes.data, index.ctypes.data, counts.ctypes.data),
           "sinet_compile_prefix_table")
    return {"nets": nets[: counts[0]], "len_offset": off, "lo": lo[: counts[1]],
            "hi": hi[: counts[1]], "index": index, "n_unique": int(counts[0]),
            "n_intervals": int(counts[1]), "index_bits": int(counts[2]),
            "max_range": int(counts[3])}


LAYOUT_KEYS = ("off_blocks", "off_desc", "desc_bits", "iv_bytes", "off_nets", "off_groups",
               "n_groups", "pml_bytes", "off_lo", "off_hi", "off_idx32", "index_bits", "n_iv",
               "max_blocks", "iv_fits_smem", "pml_fits_smem")


def sinet_prefix_table_image(net, ln):
    """(image bytes as numpy uint8, layout dict) of the table's device image."""
    net = np.ascontiguousarray(net, np.uint32)
    ln = np.ascontiguousarray(ln, np.uint8)
    layout = np.zeros(16, np.uint32)
    size = ctypes.c_size_t()
    args = (net.ctypes.data if len(net) else None, ln.ctypes.data if len(ln) else None, len(net))
    _check(load().sinet_prefix_table_image(*args, None, 0, layout.ctypes.data, ctypes.byref(size)),
           "sinet_prefix_table_image")
    img = np.zeros(size.value, np.uint8)
    _check(load().sinet_prefix_table_image(*args, img.ctypes.data, size.value, layout.ctypes.data,
                                           ctypes.byref(size)), "sinet_prefix_table_image")
    return img, dict(zip(LAYOUT_KEYS, (int(v) for v in layout)))


def sinet_build_prefix_table(net, ln, stream=None) -> int:
    net = np.ascontiguousarray(net, np.uint32)
    ln = np.ascontiguousarray(ln, np.uint8)
    h = ctypes.c_void_p()
    _check(load().sinet_build_prefix_table(net.ctypes.data if len(net) else None,
                                           ln.ctypes.data if len(ln) else None, len(net),
                                           _stream(stream), ctypes.byref(h)),
           "sinet_build_prefix_table")
    return int(h.value)


def sinet_destroy_prefix_table(handle: int):
    _check(load().sinet_destroy_prefix_table(handle), "sinet_destroy_prefix_table")


def sinet_discriminate(table: int, d_src, d_dst, n: int, d_class, d_class_counts,
                       lookup: int = LOOKUP_AUTO, stream=None):
    _check(load().sinet_discriminate(table, _dptr(d_src), _dptr(d_dst), n, _dptr(d_class),
                                     _dptr(d_class_counts), lookup, _stream(stream)),
           "sinet_discriminate")


def sinet_bin(d_ts, n: int, t0_ms: int, bin_width_ms: int, n_bins: int, d_bin, stream=None):
    _check(load().sinet_bin(_dptr(d_ts), n, t0_ms, bin_width_ms, n_bins, _dptr(d_bin), _stream(stream)),
           "sinet_bin")


def sinet_histogram(d_ts, d_bytes, d_class, n: int, params: HistParamsC, out: HistOutC, stream=None):
    _check(load().sinet_histogram(_dptr(d_ts), _dptr(d_bytes), _dptr(d_class), n,
                                  ctypes.byref(params), ctypes.byref(out), _stream(stream)),
           "sinet_histogram")


def sinet_discriminate_histogram(table: int, d_ts, d_src, d_dst, d_bytes, n: int,
                                 params: HistParamsC, out: HistOutC, stream=None):
    _check(load().sinet_discriminate_histogram(table, _dptr(d_ts), _dptr(d_src), _dptr(d_dst),
                                               _dptr(d_bytes), n, ctypes.byref(params),
                                               ctypes.byref(out), _stream(stream)),
           "sinet_discriminate_histogram")


def sinet_discriminate_histogram_noalloc(table: int, d_ts, d_src, d_dst, d_bytes, n: int,
                                         params: HistParamsC, out: HistOutC, stream=None):
    """The allocation-free plain path (fixed device scratch; see include/sinet.h)."""
    _check(load().sinet_discriminate_histogram_noalloc(table, _dptr(d_ts), _dptr(d_src), _dptr(d_dst),
                                                       _dptr(d_bytes), n, ctypes.byref(params),
                                                       ctypes.byref(out), _stream(stream)),
           "sinet_discriminate_histogram_noalloc")


def sinet_device_status(stream=None) -> int:
    v = ctypes.c_uint32()
    _check(load().sinet_device_status(_stream(stream), ctypes.byref(v)), "sinet_device_status")
    return int(v.value)


def sinet_histogram_rollup(inp: HistOutC, n_bins: int, factor: int, accumulate: bool, out: HistOutC,
                           stream=None):
    _check(load().sinet_histogram_rollup(ctypes.byref(inp), n_bins, factor, int(accumulate),
                                         ctypes.byref(out), _stream(stream)), "sinet_histogram_rollup")


def sinet_histogram_sparse(inp: HistOutC, n_bins: int, d_bin, d_count0, d_count1, d_bytes0, d_bytes1,
                           cap: int, d_n_out, stream=None):
    _check(load().sinet_histogram_sparse(ctypes.byref(inp), n_bins, _dptr(d_bin), _dptr(d_count0),
                                         _dptr(d_count1), _dptr(d_bytes0), _dptr(d_bytes1), cap,
                                         _dptr(d_n_out), _stream(stream)), "sinet_histogram_sparse")


def sinet_batch_create(slices, flags: int = 0, stream=None) -> int:
    """``slices``: a sequence of BatchSliceC (kept alive by the caller)."""
    arr = (BatchSliceC * len(slices))(*slices)
    h = ctypes.c_void_p()
    _check(load().sinet_batch_create(arr, len(slices), flags, _stream(stream), ctypes.byref(h)),
           "sinet_batch_create")
    return int(h.value)


def sinet_batch_run(handle: int, stream=None):
    _check(load().sinet_batch_run(handle, _stream(stream)), "sinet_batch_run")


def sinet_batch_strategy(handle: int, i: int) -> int:
    v = ctypes.c_int32()
    _check(load().sinet_batch_strategy(handle, i, ctypes.byref(v)), "sinet_batch_strategy")
    return int(v.value)


def sinet_batch_info(handle: int):
    items, records = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().sinet_batch_info(handle, ctypes.byref(items), ctypes.byref(records)),
           "sinet_batch_info")
    return int(items.value), int(records.value)


def sinet_batch_destroy(handle: int):
    _check(load().sinet_batch_destroy(handle), "sinet_batch_destroy")


# ---------------------------------------------------------------------------
# Conveniences


class PrefixTable:
    """A compiled CIDR list on the current device."""

    def __init__(self, net, ln, stream=None):
        self.net = np.ascontiguousarray(net, np.uint32)
        self.ln = np.ascontiguousarray(ln, np.uint8)
        self.handle = sinet_build_prefix_table(self.net, self.ln, stream)

    def close(self):
        if getattr(self, "handle", None):
            sinet_destroy_prefix_table(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class HistParams:
    t0_ms: int
    bin_width_ms: int
    n_bins: int
    policy: tuple = EXCLUSIVE
    accumulate: bool = False
    strategy: str | int = "auto"
    lookup: str | int = "auto"
    hints: int = 0
    tile_bins: int = 0
    block_threads: int = 0
    watch: object = None  # PrefixTable: only records with src or dst in it are binned

    def c(self) -> HistParamsC:
        p = HistParamsC()
        p.t0_ms, p.bin_width_ms, p.n_bins = self.t0_ms, self.bin_width_ms, self.n_bins
        for i in range(4):
            p.policy[i] = self.policy[i]
        p.accumulate = int(bool(self.accumulate))
        p.strategy = STRATEGIES[self.strategy] if isinstance(self.strategy, str) else self.strategy
        p.lookup = LOOKUPS[self.lookup] if isinstance(self.lookup, str) else self.lookup
        p.hints, p.tile_bins, p.block_threads = self.hints, self.tile_bins, self.block_threads
        p.watch = self.watch.handle if self.watch is not None else None
        return p


class Histogram:
    """Device outputs: count[2, n_bins] (uint32 bits in int32), bytes[2, n_bins]
    (uint64 bits in int64) and stats[8] (uint64 bits in int64)."""

    def __init__(self, n_bins: int, device=None, zero: bool = True):
        import torch

        device = device or torch.device("cuda")
        mk = torch.zeros if zero else torch.empty
        self.n_bins = n_bins
        self.count = mk((2, n_bins), dtype=torch.int32, device=device)
        self.bytes = mk((2, n_bins), dtype=torch.int64, device=device)
        self.stats = mk(8, dtype=torch.int64, device=device)

    def c(self) -> HistOutC:
        o = HistOutC()
        o.count[0] = self.count[0].data_ptr()
        o.count[1] = self.count[1].data_ptr()
        o.bytes[0] = self.bytes[0].data_ptr()
        o.bytes[1] = self.bytes[1].data_ptr()
        o.stats = self.stats.data_ptr()
        return o

    def to_numpy(self) -> dict:
        return {"count": self.count.cpu().numpy().view(np.uint32),
                "bytes": self.bytes.cpu().numpy().view(np.uint64),
                "stats": self.stats.cpu().numpy().view(np.uint64)}


def discriminate(table: PrefixTable, src, dst, cls=None, lookup="auto", stream=None):
    """Class counts (uint64[4] bits in an int64 CUDA tensor); class bytes into ``cls``."""
    import torch

    counts = torch.empty(4, dtype=torch.int64, device=src.device)
    sinet_discriminate(table.handle, src, dst, src.numel(), cls, counts,
                       LOOKUPS[lookup] if isinstance(lookup, str) else lookup, stream)
    return counts


def histogram(ts, nbytes, cls, params: HistParams, out: Histogram, stream=None):
    sinet_histogram(ts, nbytes, cls, ts.numel(), params.c(), out.c(), stream)
    return out


def auto_strategy(table: "PrefixTable", n: int, params: "HistParams") -> str:
    """The strategy AUTO would run for n records with these parameters."""
    v = ctypes.c_int32()
    _check(load().sinet_auto_strategy(table.handle, n, ctypes.byref(params.c()), ctypes.byref(v)),
           "sinet_auto_strategy")
    return next(k for k, x in STRATEGIES.items() if x == v.value)


def bin_index(ts, t0_ms: int, bin_width_ms: int, n_bins: int, out=None, stream=None):
    """Bin of each timestamp (uint32 bits in int32; 0xFFFFFFFF outside the window)."""
    import torch

    out = out if out is not None else torch.empty(ts.numel(), dtype=torch.int32, device=ts.device)
    sinet_bin(ts, ts.numel(), t0_ms, bin_width_ms, n_bins, out, stream)
    return out


def discriminate_histogram(table: PrefixTable, ts, src, dst, nbytes, params: HistParams,
                           out: Histogram, stream=None):
    sinet_discriminate_histogram(table.handle, ts, src, dst, nbytes, ts.numel(), params.c(),
                                 out.c(), stream)
    return out


class Batch:
    """A batch of independent slices run by one persistent graph-captured launch.

    ``slices``: sequence of (table: PrefixTable, ts, src, dst, nbytes, params:
    HistParams, out: Histogram). The tensors, tables and outputs are referenced
    by the batch and kept alive here."""

    def __init__(self, slices, autotune: bool = False, stream=None, ready=None):
        """``ready``: optional per-slice (device uint32 tensor view of one word, value) or None."""
        self._keep = list(slices)
        self._ready = list(ready) if ready is not None else [None] * len(self._keep)
        cs = []
        for (table, ts, src, dst, nb, params, out), rd in zip(self._keep, self._ready):
            c = BatchSliceC()
            if rd is not None:
                c.ready, c.ready_value = _dptr(rd[0]), rd[1]
            c.ts, c.src, c.dst, c.bytes = _dptr(ts), _dptr(src), _dptr(dst), _dptr(nb)
            c.n = ts.numel()
            c.table = table.handle
            c.params = params.c()
            c.out = out.c()
            cs.append(c)
        self.handle = sinet_batch_create(cs, BATCH_AUTOTUNE if autotune else 0, stream)

    def run(self, stream=None):
        sinet_batch_run(self.handle, stream)

    def set_wait(self, wait_ns: int):
        _check(load().sinet_batch_set_wait(self.handle, wait_ns), "sinet_batch_set_wait")

    def strategy(self, i: int) -> str:
        v = sinet_batch_strategy(self.handle, i)
        return next(k for k, x in STRATEGIES.items() if x == v)

    def info(self):
        return sinet_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sinet_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _hptr(a) -> int | None:
    """Host address of a numpy array or CPU tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a contiguous array")
        return a.ctypes.data
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("expected a contiguous CPU tensor")
    return a.data_ptr()


class Server:
    """Continuous-batching serving loop (C ABI sinet_server_*).

    ``tenants``: sequence of (PrefixTable, HistParams); each tenant keeps a
    resident histogram that its requests accumulate into. Host record
    buffers of a request are kept alive here until it is waited for."""

    def __init__(self, tenants, budget_bytes: int = 1 << 30, max_requests_per_launch: int = 256,
                 max_queued: int = 1 << 20):
        self._tables = [t for t, _ in tenants]
        self.n_bins = [p.n_bins for _, p in tenants]
        arr = (TenantC * len(tenants))()
        for i, (t, p) in enumerate(tenants):
            arr[i].table = t.handle
            arr[i].params = p.c()
        cfg = ServerConfigC(budget_bytes, max_requests_per_launch, max_queued)
        h = ctypes.c_void_p()
        _check(load().sinet_server_create(ctypes.byref(cfg), arr, len(tenants), ctypes.byref(h)),
               "sinet_server_create")
        self.handle = int(h.value)
        self._keep = {}

    def submit(self, tenant: int, ts, src, dst, nbytes) -> int:
        t = ctypes.c_uint64()
        n = len(ts)
        _check(load().sinet_server_submit(self.handle, tenant, _hptr(ts), _hptr(src), _hptr(dst),
                                          _hptr(nbytes), n, ctypes.byref(t)), "sinet_server_submit")
        self._keep[int(t.value)] = (ts, src, dst, nbytes)
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = 120_000) -> dict:
        info = RequestInfoC()
        _check(load().sinet_server_wait(self.handle, ticket, timeout_ms, ctypes.byref(info)),
               "sinet_server_wait")
        self._keep.pop(ticket, None)
        return {"n": int(info.n), "launch": int(info.launch), "latency_ns": int(info.latency_ns)}

    def drain(self, timeout_ms: int = 600_000):
        _check(load().sinet_server_drain(self.handle, timeout_ms), "sinet_server_drain")

    def export(self, tenant: int) -> dict:
        nb = self.n_bins[tenant]
        c = np.zeros((2, nb), np.uint32)
        b = np.zeros((2, nb), np.uint64)
        st = np.zeros(8, np.uint64)
        _check(load().sinet_server_export(self.handle, tenant, c.ctypes.data, b.ctypes.data,
                                          st.ctypes.data), "sinet_server_export")
        return {"count": c, "bytes": b, "stats": st}

    def import_(self, tenant: int, hist: dict):
        """Replace a tenant's resident histogram with {"count", "bytes", "stats"} host arrays."""
        c = np.ascontiguousarray(hist["count"], np.uint32)
        b = np.ascontiguousarray(hist["bytes"], np.uint64)
        st = np.ascontiguousarray(hist["stats"], np.uint64)
        assert c.shape == (2, self.n_bins[tenant]) and b.shape == c.shape and st.shape == (8,)
        _check(load().sinet_server_import(self.handle, tenant, c.ctypes.data, b.ctypes.data,
                                          st.ctypes.data), "sinet_server_import")

    def stats(self, reset: bool = False) -> dict:
        c = ServerCountersC()
        _check(load().sinet_server_stats(self.handle, int(reset), ctypes.byref(c)), "sinet_server_stats")
        return {k: int(getattr(c, k)) for k, _ in ServerCountersC._fields_}

    def close(self):
        if getattr(self, "handle", None):
            _check(load().sinet_server_destroy(self.handle), "sinet_server_destroy")
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rollup(hist: "Histogram", factor: int, out: "Histogram | None" = None, accumulate: bool = False,
           stream=None) -> "Histogram":
    """Coarser bins: out bin j sums bins [j * factor, (j + 1) * factor)."""
    n_out = -(-hist.n_bins // factor)
    out = out or Histogram(n_out, hist.count.device, zero=False)
    sinet_histogram_rollup(hist.c(), hist.n_bins, factor, accumulate, out.c(), stream)
    return out


def sparse(hist: "Histogram", cap: int | None = None, stream=None) -> dict:
    """Non-empty bins in order: {"n": total, "bin", "count" [2, k], "bytes" [2, k]} (device
    tensors; k = min(total, cap))."""
    import torch

    dev = hist.count.device
    cap = hist.n_bins if cap is None else cap
    b = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    c = torch.empty((2, max(cap, 1)), dtype=torch.int32, device=dev)
    y = torch.empty((2, max(cap, 1)), dtype=torch.int64, device=dev)
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    sinet_histogram_sparse(hist.c(), hist.n_bins, b, c[0], c[1], y[0], y[1], cap, n, stream)
    total = int(n.item())
    k = min(total, cap)
    return {"n": total, "bin": b[:k], "count": c[:, :k], "bytes": y[:, :k]}
