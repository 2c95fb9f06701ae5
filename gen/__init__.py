"""Seeded synthetic workloads for the session-discrimination hot path.

Shapes only: prefix tables, SoA session records (ts_ms u64, src_ip u32,
dst_ip u32, bytes u32) and batch/serving request streams, after the paper's
workloads (Table 1 fields 1, 5, 8 and 21; Table 2's daily volumes; the diurnal
pattern of Figs. 6-7). Holds none of the method's arithmetic: no membership
test, no binning, no counting. The C side lives in ``sinet_gen.c``; the
shared library is compiled by ``__graft_entry__.build()`` into ``gen/_lib``.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsinet_gen.so")
SOURCE = os.path.join(_HERE, "sinet_gen.c")

DAY_MS = 86_400_000
BASE_SEED = 2106128630


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_total", ctypes.c_uint64),
        ("class_p", ctypes.c_double * 4),
        ("bytes_mu", ctypes.c_double),
        ("bytes_sigma", ctypes.c_double),
        ("ts_kind", ctypes.c_int32),
        ("host_kind", ctypes.c_int32),
        ("t_lo", ctypes.c_uint64),
        ("t_hi", ctypes.c_uint64),
        ("jitter", ctypes.c_uint64),
        ("peak_frac", ctypes.c_double),
        ("zipf_s", ctypes.c_double),
        ("zipf_bins", ctypes.c_uint64),
        ("zipf_w", ctypes.c_uint64),
        ("pool_size", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        L.gen_table.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_int, P, P]
        L.gen_table.restype = ctypes.c_int
        L.gen_records.argtypes = [ctypes.POINTER(_Params), P, P, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_uint64, P, P, P, P, P]
        L.gen_records.restype = ctypes.c_int
        L.gen_zipf.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                               ctypes.c_uint64, P]
        L.gen_zipf.restype = ctypes.c_uint64
        L.gen_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, P]
        L.gen_u64.restype = None
        L.gen_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return int(a.data_ptr())  # torch tensor on the host (pinned or not)


# --------------------------------------------------------------------------
# Tables


@dataclass(frozen=True)
class TableSpec:
    n: int
    len_lo: int
    len_hi: int
    weighted: bool = False


def make_table(spec: TableSpec, seed: int):
    """Return (net u32[n], len u8[n]); networks inside 0.0.0.0/1, host bits clear."""
    net = np.empty(spec.n, np.uint32)
    ln = np.empty(spec.n, np.uint8)
    rc = lib().gen_table(seed, spec.n, spec.len_lo, spec.len_hi, int(spec.weighted),
                         _ptr(net), _ptr(ln))
    if rc != 0:
        raise ValueError(f"bad table spec {spec}")
    return net, ln


# --------------------------------------------------------------------------
# Records


@dataclass(frozen=True)
class RecordSpec:
    n: int
    class_p: tuple = (0.10, 0.40, 0.40, 0.10)  # neither, src inside, dst inside, both
    bytes_mu: float = 8.0
    bytes_sigma: float = 2.0
    ts_kind: str = "uniform"  # uniform | diurnal | zipf
    host_kind: str = "prefix"  # prefix | zipf
    t_lo: int = 0
    t_hi: int = 3_600_000
    jitter: int = 500
    peak_frac: float = 14.0 / 24.0
    zipf_s: float = 1.1
    zipf_bins: int = DAY_MS
    zipf_w: int = 1
    pool_size: int = 25_000


_TS_KIND = {"uniform": 0, "diurnal": 1, "zipf": 2}
_HOST_KIND = {"prefix": 0, "zipf": 1}


def _params(spec: RecordSpec, seed: int) -> _Params:
    p = _Params()
    p.seed = seed
    p.n_total = spec.n
    for i in range(4):
        p.class_p[i] = spec.class_p[i]
    p.bytes_mu = spec.bytes_mu
    p.bytes_sigma = spec.bytes_sigma
    p.ts_kind = _TS_KIND[spec.ts_kind]
    p.host_kind = _HOST_KIND[spec.host_kind]
    p.t_lo = spec.t_lo
    p.t_hi = spec.t_hi
    p.jitter = spec.jitter
    p.peak_frac = spec.peak_frac
    p.zipf_s = spec.zipf_s
    p.zipf_bins = spec.zipf_bins
    p.zipf_w = spec.zipf_w
    p.pool_size = spec.pool_size
    return p


def fill_records(spec: RecordSpec, seed: int, net, ln, first: int, n: int,
                 ts=None, src=None, dst=None, nbytes=None, intended_class=None):
    """Write records [first, first+n) of the workload into caller buffers
    (numpy arrays or host torch tensors, any may be None)."""
    p = _params(spec, seed)
    rc = lib().gen_records(ctypes.byref(p), _ptr(net), _ptr(ln), len(net), first, n,
                           _ptr(ts), _ptr(src), _ptr(dst), _ptr(nbytes), _ptr(intended_class))
    if rc != 0:
        raise ValueError("gen_records rejected its arguments")


def make_records(spec: RecordSpec, seed: int, net, ln, first: int = 0, n: int | None = None,
                 with_class: bool = False):
    """Numpy SoA records [first, first+n) (default: the whole workload)."""
    n = spec.n - first if n is None else n
    ts = np.empty(n, np.uint64)
    src = np.empty(n, np.uint32)
    dst = np.empty(n, np.uint32)
    nb = np.empty(n, np.uint32)
    ic = np.empty(n, np.uint8) if with_class else None
    fill_records(spec, seed, net, ln, first, n, ts, src, dst, nb, ic)
    out = {"ts": ts, "src": src, "dst": dst, "bytes": nb}
    if with_class:
        out["intended_class"] = ic
    return out


def zipf_ranks(s: float, n: int, seed: int, count: int, first: int = 0):
    out = np.empty(count, np.uint64)
    lib().gen_zipf(s, n, seed, first, count, _ptr(out))
    return out


def u64_stream(seed: int, stream: int, n: int, first: int = 0):
    out = np.empty(n, np.uint64)
    lib().gen_u64(seed, stream, first, n, _ptr(out))
    return out


def threads() -> int:
    return int(lib().gen_num_threads())


# --------------------------------------------------------------------------
# The five workloads (record counts, tables, bins).


@dataclass(frozen=True)
class Workload:
    name: str
    table: TableSpec
    records: RecordSpec
    t0: int
    bin_width: int
    n_bins: int
    seed: int
    note: str = ""


WORKLOADS = {
    # plain method, tiny: 1 M records over one hour, 64 prefixes /16-/24
    "tiny": Workload(
        "tiny-1M-uniform-1h", TableSpec(64, 16, 24),
        RecordSpec(1_000_000, ts_kind="uniform", t_lo=0, t_hi=3_600_000),
        t0=0, bin_width=1, n_bins=3_600_000, seed=BASE_SEED + 1),
    # one paper-scale day: 400 M time-sorted records, diurnal 3:1, +-500 ms jitter
    "day": Workload(
        "day-400M-diurnal-sorted", TableSpec(2000, 8, 30, weighted=True),
        RecordSpec(400_000_000, ts_kind="diurnal", t_lo=0, t_hi=DAY_MS, jitter=500),
        t0=0, bin_width=1, n_bins=DAY_MS, seed=BASE_SEED + 2),
    # heavy day: 1.6 B unsorted records, Zipf(1.1) bins and hosts, 8,000 prefixes /8-/32
    "heavy": Workload(
        "heavy-1.6B-zipf-unsorted", TableSpec(8000, 8, 32),
        RecordSpec(1_600_000_000, ts_kind="zipf", host_kind="zipf", t_lo=0, t_hi=DAY_MS,
                   zipf_bins=DAY_MS, zipf_w=1, pool_size=25_000),
        t0=0, bin_width=1, n_bins=DAY_MS, seed=BASE_SEED + 3),
}


def scaled(w: Workload, n: int) -> Workload:
    """The same workload shape with n records (sorted kinds keep their day)."""
    return replace(w, records=replace(w.records, n=n))


# --------------------------------------------------------------------------
# Batched slices (256 uneven slices, each with its own window, width, table)


@dataclass
class SliceSpec:
    index: int
    n: int
    t0: int
    window: int
    bin_width: int
    n_bins: int
    table: TableSpec
    seed: int
    records: RecordSpec = field(default=None)


def batch_slices(n_slices: int = 256, seed: int = BASE_SEED + 4, n_lo: int = 10_000,
                 n_hi: int = 20_000_000, scale: float = 1.0):
    """Slice plan: sizes log-uniform in [n_lo, n_hi] (times ``scale``), windows
    log-uniform 1 min - 6 h, bin width in {1, 10, 1000} ms, tables of
    16-4,000 prefixes (log-uniform) with lengths /8-/32."""
    r = u64_stream(seed, 1, 8 * n_slices).reshape(n_slices, 8)
    u = (r >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    out = []
    for i in range(n_slices):
        n = int(math.exp(math.log(n_lo) + u[i, 0] * (math.log(n_hi) - math.log(n_lo))) * scale)
        n = max(n, 1)
        window = int(math.exp(math.log(60_000) + u[i, 1] * (math.log(21_600_000) - math.log(60_000))))
        w = (1, 10, 1000)[min(int(u[i, 2] * 3), 2)]
        n_bins = -(-window // w)
        t0 = int(u[i, 3] * (DAY_MS - window))
        P = int(math.exp(math.log(16) + u[i, 4] * (math.log(4000) - math.log(16))))
        tspec = TableSpec(P, 8, 32)
        rspec = RecordSpec(n, ts_kind="uniform", t_lo=t0, t_hi=t0 + window)
        out.append(SliceSpec(i, n, t0, window, w, n_bins, tspec, seed * 1000 + i, rspec))
    return out


# --------------------------------------------------------------------------
# Serving stream (tenants with their own tables; Poisson arrivals; log-normal
# request sizes; each request uniform over a random window of its tenant's day)


@dataclass
class RequestSpec:
    index: int
    tenant: int
    n: int
    gap: float  # exponential(1) inter-arrival gap, scaled by 1 / rate by the caller
    seed: int
    records: RecordSpec


def serving_plan(n_tenants: int = 32, n_requests: int = 1000, seed: int = BASE_SEED + 5,
                 median: float = 1_000_000, sigma: float = math.log(50) / 2.326,
                 cap: int | None = None, p_lo: int = 500, p_hi: int = 4000):
    """(tenant table specs, request specs). Request sizes are log-normal with the
    given median and sigma (p99 = 50 x median by default), capped at ``cap``;
    windows are log-uniform 1 min - 6 h at a uniform start within the day."""
    t = u64_stream(seed, 1, n_tenants)
    tables = [TableSpec(p_lo + int((int(x) >> 11) * 2.0 ** -53 * (p_hi - p_lo + 1)), 8, 32) for x in t]
    r = u64_stream(seed, 2, 6 * n_requests).reshape(n_requests, 6)
    u = ((r >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    out = []
    for i in range(n_requests):
        z = math.sqrt(-2.0 * math.log(u[i, 0])) * math.cos(2.0 * math.pi * u[i, 1])  # Box-Muller
        n = max(1, int(median * math.exp(sigma * z)))
        if cap:
            n = min(n, cap)
        tenant = min(int(u[i, 2] * n_tenants), n_tenants - 1)
        window = int(math.exp(math.log(60_000) + u[i, 3] * (math.log(21_600_000) - math.log(60_000))))
        t_lo = int(u[i, 4] * (DAY_MS - window))
        gap = -math.log(u[i, 5])
        out.append(RequestSpec(i, tenant, n, gap, seed * 1000 + i,
                               RecordSpec(n, ts_kind="uniform", t_lo=t_lo, t_hi=t_lo + window)))
    return tables, out
