"""Benchmark: discriminate + millisecond-histogram a paper-scale day on GB300.

Default workload: the heavy day, 1.6 B unsorted session records whose bins
and hosts are Zipf(1.1)-skewed, 8,000 CIDR prefixes /8-/32, 1 ms bins over
24 h (86.4 M bins x 2 directions). A step = one fused discriminate/histogram
call over all records (plus the output zeroing for the strategies that need
it; inputs resident in HBM, 32 GB of records, far larger than L2). The
strategy is picked by one timed run of each candidate. The plain
discriminate -> radix sort -> reduce-by-key path is timed on the same data
for comparison, ``e2e`` times the same step through the public API with the
records copied from pinned host memory and the histogram copied back every
step, and the 400 M-record time-sorted day (2,000 prefixes) is timed as a
second line of figures under ``day``.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload heavy|day|tiny|batch|serve]
                  [--shard replicas|records|time]
  python bench.py --impl reference ...   # the CPU oracle on the host cores

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gen  # noqa: E402

METRIC = "sessions/sec (bit-exact) and HBM GB/s vs peak, fused vs sort+reduce on 1 GB300"
UNIT = "sessions/s"
RECORD_BYTES = 20   # ts u64 + src u32 + dst u32 + bytes u32
BIN_BYTES = 24      # 2 directions x (u32 count + u64 byte sum)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="heavy", choices=sorted(gen.WORKLOADS) + ["batch", "serve"],
                    help="heavy | day | tiny: one window; batch: 256 uneven slices in one "
                         "persistent launch; serve: the continuous-batching serving loop")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "records", "time"],
                    help="with N > 1 ranks: replicas (every rank its own workload, weak scaling); "
                         "records (one workload split by record range, partial histograms merged by "
                         "an NCCL reduce-scatter inside the timed step; strong); time (one "
                         "time-sorted workload split by owned bin range, no collective; strong)")
    ap.add_argument("--no-day", action="store_true",
                    help="heavy: skip the extra line of figures for the time-sorted 400 M day")
    ap.add_argument("--slices", type=int, default=256, help="batch: number of slices")
    ap.add_argument("--tenants", type=int, default=32, help="serve: tenants")
    ap.add_argument("--requests", type=int, default=2000, help="serve: requests per phase")
    ap.add_argument("--request-cap", type=int, default=16_000_000,
                    help="serve: largest request (records); sizes above it are capped")
    ap.add_argument("--budget-gb", type=float, default=40.0, help="serve: in-flight arena")
    ap.add_argument("--records", type=int, default=0, help="override the record count")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink records, window and bins together (keeps records per bin; "
                         "for profiling captures)")
    ap.add_argument("--strategy", default="tune",
                    help="tune | partition | owner | global_atomic | priv_tile | atomic_noagg | atomic_cell "
                         "| sort_reduce")
    ap.add_argument("--plain-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-post", action="store_true", help="skip the roll-up / sparse timings")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def max_over_ranks(x: float, device) -> float:
    """The slowest rank's value (the job's time): an all-reduce MAX when a
    process group is up, else x."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: the units every rank processed, over the slowest rank's time."""
    return world * units_per_rank * steps / (total_ms / 1e3)


def rank_seed(base: int, rank: int, stride: int = 1) -> int:
    """Weak scaling: each rank draws its own workload (different seed, same shape)."""
    return base + stride * rank


def data_digest(tensors, sample: int = 1 << 20) -> str:
    """SHA-256 over the first `sample` elements of each host buffer (a
    reproducibility stamp of the generated input)."""
    h = hashlib.sha256()
    for t in tensors:
        h.update(t[:sample].numpy().tobytes())
    return h.hexdigest()[:16]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_named(name):
    return gen.WORKLOADS[name]


def owned_records(w, net, ln, world, rank, chunk=50_000_000):
    """Time-range split: the records of workload w whose ts falls in this
    rank's owned bins (rank 0 also takes the records outside the window),
    generated chunk by chunk and kept in pinned host memory."""
    import torch

    from paper_2106_12863_gb300 import shard

    win = shard.Window(w.t0, w.bin_width, w.n_bins).owned(world, rank)
    lo, hi = win.t0, win.t0 + win.n_bins * win.width
    end = w.t0 + w.n_bins * w.bin_width
    parts = {k: [] for k in ("ts", "src", "dst", "bytes")}
    for first in range(0, w.records.n, chunk):
        r = gen.make_records(w.records, w.seed, net, ln, first=first, n=min(chunk, w.records.n - first))
        keep = (r["ts"] >= np.uint64(lo)) & (r["ts"] < np.uint64(hi))
        if rank == 0:
            keep |= (r["ts"] < np.uint64(w.t0)) | (r["ts"] >= np.uint64(end))
        for k in parts:
            parts[k].append(r[k][keep])
    out = {}
    for k, dt in (("ts", torch.int64), ("src", torch.int32), ("dst", torch.int32), ("bytes", torch.int32)):
        a = np.concatenate(parts[k])
        t = torch.empty(len(a), dtype=dt, pin_memory=True)
        t.numpy()[:] = a.view(t.numpy().dtype)
        out[k] = t
    return out


def workload(args, rank):
    from dataclasses import replace

    w = gen.WORKLOADS[args.workload]
    if args.records:
        w = gen.scaled(w, args.records)
    if args.scale != 1.0:
        f = args.scale
        r = w.records
        span = int((r.t_hi - r.t_lo) * f)
        rec = replace(r, n=int(r.n * f), t_hi=r.t_lo + span,
                      zipf_bins=max(1, int(r.zipf_bins * f)))
        w = replace(w, records=rec, n_bins=max(1, int(w.n_bins * f)),
                    name=f"{w.name}-scale{f:g}")
    return w


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# The files each timed kernel is compiled from: its translation unit and the
# headers it includes.
KERNEL_SOURCES = {
    "k_fused_tile": ["fused.cu", "combine.cuh", "launch.h", "records.cuh", "common.cuh"],
    "k_fused_atomic": ["fused.cu", "combine.cuh", "launch.h", "records.cuh", "common.cuh"],
    "k_fused_owner": ["owner.cu", "owner.h", "launch.h", "records.cuh", "common.cuh"],
    "k_part_main": ["partition.cu", "partition.h", "combine.cuh", "launch.h", "records.cuh", "common.cuh"],
}


def _code_only(text: str) -> str:
    """Source text without comments or layout: a comment edit leaves it as is."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(kernel: str | None = None):
    """Hash of a kernel's source code (all of csrc/ for other kernels),
    comments and whitespace excluded."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2106_12863_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) or sorted(
        f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh", ".h", ".cpp")))
    for f in files:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(f.encode())
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash(kernel)
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = dict(kv.split("=", 1) for kv in line.split())
            if parts.get("kernel") == kernel and parts.get("workload") == workload \
                    and parts.get("source") == cur:
                return float(parts["bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(index), "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        self.window = (None, None)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, start: bool):
        t = time.time()
        a, b = self.window
        self.window = (t, b) if start else (a, t)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        a, b = self.window
        rows = [ln for t, ln in self.lines if a is not None and a - 0.15 <= t <= b + 0.15]
        if not rows:
            rows = [ln for _, ln in self.lines[-3:]]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, seconds: float):
    """The oracle, as it stands, on a bounded sample of the workload."""
    import oracle

    o = oracle.get()
    net, ln = gen.make_table(w.table, w.seed)
    mid = w.records.n // 2
    probe = min(100_000, w.records.n)
    rec = gen.make_records(w.records, w.seed, net, ln, first=mid - probe // 2, n=probe)
    t = time.perf_counter()
    o.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, min(w.n_bins, 1 << 27))
    dt = time.perf_counter() - t
    m = int(min(w.records.n, max(probe, probe * seconds / max(dt, 1e-6))))
    rec = gen.make_records(w.records, w.seed, net, ln, first=max(0, mid - m // 2), n=m)
    t = time.perf_counter()
    o.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    dt = time.perf_counter() - t
    return {"value": m / dt, "unit": UNIT, "cores": o.threads(), "kind": "oracle",
            "sample": f"{m} contiguous records from the middle of the {w.name} workload, "
                      f"full {w.table.n}-prefix table, {w.n_bins} bins; {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    o = oracle.get()
    if args.workload in ("batch", "serve"):
        run_reference_batch(args, o)
        return
    w = workload(args, rank)
    net, ln = gen.make_table(w.table, w.seed)
    # size each step's sample so that all warm-up + timed steps fit ~2.5 minutes
    per_step = max(0.05, 150.0 / (args.steps + args.warmup))
    probe = min(50_000, w.records.n)
    rec = gen.make_records(w.records, w.seed, net, ln, n=probe)
    t = time.perf_counter()
    o.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
    dt = time.perf_counter() - t
    m = int(min(w.records.n, max(1000, probe * per_step / max(dt, 1e-6))))
    samples = []
    for s in range(args.warmup + args.steps):
        first = (s * m) % max(1, w.records.n - m)
        rec = gen.make_records(w.records, w.seed, net, ln, first=first, n=m)
        t = time.perf_counter()
        o.discriminate_histogram(net, ln, rec, w.t0, w.bin_width, w.n_bins)
        if s >= args.warmup:
            samples.append(time.perf_counter() - t)
    total = sum(samples)
    value = m * len(samples) / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(samples),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "records_per_step": m, "prefixes": w.table.n,
                       "n_bins": w.n_bins},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.threads(), "kind": "oracle",
                             "sample": f"{m} records of {w.name} per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class _OutView:
    """Histogram outputs of one batch slice: views into flat device arrays."""

    def __init__(self, count, nbytes, stats, off, nb, i):
        self.count = count[2 * off: 2 * off + 2 * nb].view(2, nb)
        self.bytes = nbytes[2 * off: 2 * off + 2 * nb].view(2, nb)
        self.stats = stats[i]

    def c(self):
        import paper_2106_12863_gb300 as sinet

        o = sinet.HistOutC()
        o.count[0], o.count[1] = self.count[0].data_ptr(), self.count[1].data_ptr()
        o.bytes[0], o.bytes[1] = self.bytes[0].data_ptr(), self.bytes[1].data_ptr()
        o.stats = self.stats.data_ptr()
        return o


def run_batch_bench(args):
    """256 uneven slices (own table, window, bin width each) as one batch:
    the graph-captured persistent launch against one call per slice (fused and
    plain)."""
    rank, world, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    import paper_2106_12863_gb300 as sinet

    sinet.load()
    plan = gen.batch_slices(n_slices=args.slices, seed=rank_seed(gen.BASE_SEED + 4, rank, 1000),
                            scale=args.scale)
    n_tot = sum(sp.n for sp in plan)
    bins_tot = sum(sp.n_bins for sp in plan)
    tg = time.perf_counter()
    h = {"ts": torch.empty(n_tot, dtype=torch.int64, pin_memory=True),
         "src": torch.empty(n_tot, dtype=torch.int32, pin_memory=True),
         "dst": torch.empty(n_tot, dtype=torch.int32, pin_memory=True),
         "bytes": torch.empty(n_tot, dtype=torch.int32, pin_memory=True)}
    tables, offs, off = [], [], 0
    for sp in plan:
        net, ln = gen.make_table(sp.table, sp.seed)
        gen.fill_records(sp.records, sp.seed, net, ln, 0, sp.n, h["ts"][off:off + sp.n],
                         h["src"][off:off + sp.n], h["dst"][off:off + sp.n], h["bytes"][off:off + sp.n])
        tables.append(sinet.PrefixTable(net, ln))
        offs.append(off)
        off += sp.n
    t_gen = time.perf_counter() - tg
    d = {k: v.to(dev) for k, v in h.items()}
    count = torch.empty(2 * bins_tot, dtype=torch.int32, device=dev)
    nbytes = torch.empty(2 * bins_tot, dtype=torch.int64, device=dev)
    stats = torch.empty((len(plan), 8), dtype=torch.int64, device=dev)
    outs, slices, boff = [], [], 0
    for i, sp in enumerate(plan):
        o = _OutView(count, nbytes, stats, boff, sp.n_bins, i)
        boff += sp.n_bins
        outs.append(o)
        a, n = offs[i], sp.n
        p = sinet.HistParams(sp.t0, sp.bin_width, sp.n_bins)
        slices.append((tables[i], d["ts"][a:a + n], d["src"][a:a + n], d["dst"][a:a + n],
                       d["bytes"][a:a + n], p, o))
    stream = torch.cuda.current_stream(dev)
    # the tuner's choices per input class (strategy, ns per record) are read
    # back from its cache file: a fresh one for this run unless the caller
    # named one
    tune_file, own_tune_file = os.environ.get("SINET_AUTOTUNE_CACHE"), False
    if not tune_file:
        import tempfile
        fd, tune_file = tempfile.mkstemp(prefix="sinet_tune_", suffix=".txt")
        os.close(fd)
        os.environ["SINET_AUTOTUNE_CACHE"] = tune_file
        own_tune_file = True
    tt = time.perf_counter()
    batch = sinet.Batch(slices, autotune=True)
    t_tune = time.perf_counter() - tt
    items, _ = batch.info()
    strat_count = {}
    for i in range(len(plan)):
        s_ = batch.strategy(i)
        strat_count[s_] = strat_count.get(s_, 0) + 1
    tuned = []
    with open(tune_file) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3:
                tuned.append({"class": parts[0], "strategy": parts[1], "ns_per_record": float(parts[2])})
    if own_tune_file:
        os.environ.pop("SINET_AUTOTUNE_CACHE", None)
        os.unlink(tune_file)

    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.mark(True)
    t_begin, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_begin.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        batch.run()
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks.mark(False)
    clk = clocks.stop()
    total_ms = t_begin.elapsed_time(t_end)
    graph_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / args.steps
    st = stats.cpu().numpy().view(np.uint64)
    for i, sp in enumerate(plan):
        assert int(st[i, :4].sum()) == sp.n, f"slice {i}: class counts do not sum to its records"
    ref_stats = st.copy()

    result = {"metric": METRIC, "value": job_rate(n_tot, world, args.steps, total_ms), "unit": UNIT,
              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "u32/u64",
              "data": "synthetic (seeded generator; 256 uneven slices)"}
    alg_bytes = RECORD_BYTES * n_tot + BIN_BYTES * bins_tot
    peak, peak_kind = peaks()
    achieved = alg_bytes / (graph_ms / 1e3) / 1e9
    result["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                          "frac": achieved / peak, "traffic": None, "kernel": "k_batch_zero + k_batch",
                          "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg_bytes,
                          "kernel_ms": graph_ms}
    result["gpu_launches"] = 2 * args.steps  # zeroing kernel + batch kernel per graph replay
    name = f"batch-{len(plan)}-slices-uneven" + (f"-scale{args.scale:g}" if args.scale != 1.0 else "")
    result["config"] = {"workload": name, "records": n_tot,
                        "slices": len(plan), "bins_total": bins_tot, "work_items": items,
                        "strategies": strat_count, "tune_s": round(t_tune, 2), "tuned_classes": tuned,
                        "l2": f"inputs larger than L2 ({RECORD_BYTES * n_tot / 1e9:.1f} GB of records)",
                        "policy": "exclusive", "parallelism": f"replicas x{world} (weak)",
                        "gen_s": round(t_gen, 1), "seed": rank_seed(gen.BASE_SEED + 4, rank, 1000),
                        "data_sha256_prefix": data_digest([h["ts"], h["src"], h["dst"], h["bytes"]])}
    result["clocks"] = clk

    def per_slice(strategy):
        for i, sp in enumerate(plan):
            t_, ts, src, dst, nb, _, o = slices[i]
            sinet.discriminate_histogram(t_, ts, src, dst, nb,
                                         sinet.HistParams(sp.t0, sp.bin_width, sp.n_bins,
                                                          strategy=strategy), o)

    for name, strategy, k in (("per_slice_fused", "auto", 3), ("per_slice_plain", "sort_reduce", 2)):
        if name == "per_slice_plain" and args.no_plain:
            continue
        per_slice(strategy)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(k):
            per_slice(strategy)
        p1.record(stream)
        torch.cuda.synchronize()
        ms = p0.elapsed_time(p1) / k
        result[name] = {"value": n_tot / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": k,
                        "launches_per_step": len(plan)}
        result[f"batched_vs_{name}"] = (n_tot / (ms_per_step / 1e3)) / result[name]["value"]
        assert np.array_equal(stats.cpu().numpy().view(np.uint64), ref_stats), name

    if not args.no_e2e:
        hout = {"count": torch.empty_like(count, device="cpu").pin_memory(),
                "bytes": torch.empty_like(nbytes, device="cpu").pin_memory(),
                "stats": torch.empty_like(stats, device="cpu").pin_memory()}

        def e2e_step():
            for k_ in d:
                d[k_].copy_(h[k_], non_blocking=True)
            batch.run()
            hout["count"].copy_(count, non_blocking=True)
            hout["bytes"].copy_(nbytes, non_blocking=True)
            hout["stats"].copy_(stats, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        q1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = q0.elapsed_time(q1) / args.e2e_steps
        result["e2e"] = {"value": world * n_tot / (e2e_ms / 1e3), "unit": UNIT,
                         "h2d_bytes_per_step": sum(v.numel() * v.element_size() for v in h.values()),
                         "d2h_bytes_per_step": sum(v.numel() * v.element_size() for v in hout.values()),
                         "ms_per_step": e2e_ms, "steps": args.e2e_steps}
        assert np.array_equal(hout["stats"].numpy().view(np.uint64), ref_stats)

    if rank == 0 and not args.no_cpu:
        import oracle

        o_ = oracle.get()
        done, t_cpu, i = 0, 0.0, 0
        while t_cpu < args.cpu_seconds and i < len(plan):
            sp = plan[i]
            net, ln = gen.make_table(sp.table, sp.seed)
            # a slice prefix at most as long as the remaining time allows at the rate so far
            cap = sp.n if done == 0 else int(done / t_cpu * (args.cpu_seconds - t_cpu)) + 1
            m = max(1, min(sp.n, cap, 200_000 if done == 0 else sp.n))
            rec = gen.make_records(sp.records, sp.seed, net, ln, n=m)
            t0_ = time.perf_counter()
            o_.discriminate_histogram(net, ln, rec, sp.t0, sp.bin_width, sp.n_bins)
            t_cpu += time.perf_counter() - t0_
            done += m
            i += 1
        result["cpu_baseline"] = {"value": done / t_cpu, "unit": UNIT, "cores": o_.threads(),
                                  "kind": "oracle",
                                  "sample": f"prefixes of the first {i} slices of the batch "
                                            f"({done} records), one oracle call per slice; "
                                            f"{t_cpu:.1f} s"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    batch.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference_batch(args, o):
    """The oracle on the batch (or serving) workload: step s runs slice (or
    request) s, cyclically, on a prefix sized so all steps fit about 2.5
    minutes."""
    if args.workload == "serve":
        specs, reqs = gen.serving_plan(n_tenants=args.tenants, n_requests=args.requests,
                                       cap=args.request_cap)
        items = [(specs[r.tenant], gen.BASE_SEED + 5000 + r.tenant, r.records, r.seed, r.n, 0, 1,
                  gen.DAY_MS) for r in reqs]
        name = f"serve-{len(specs)}-tenants-lognormal-1M"
    else:
        plan = gen.batch_slices(n_slices=args.slices)
        items = [(sp.table, sp.seed, sp.records, sp.seed, sp.n, sp.t0, sp.bin_width, sp.n_bins)
                 for sp in plan]
        name = f"batch-{len(plan)}-slices-uneven"
    per_step = max(0.05, 150.0 / (args.steps + args.warmup))
    tspec, tseed, rspec, rseed, n0, t0, w, nb = items[0]
    net, ln = gen.make_table(tspec, tseed)
    probe = min(50_000, n0)
    rec = gen.make_records(rspec, rseed, net, ln, n=probe)
    t = time.perf_counter()
    o.discriminate_histogram(net, ln, rec, t0, w, nb)
    rate = probe / max(time.perf_counter() - t, 1e-6)
    done, total = 0, 0.0
    for s in range(args.warmup + args.steps):
        tspec, tseed, rspec, rseed, n_s, t0, w, nb = items[s % len(items)]
        net, ln = gen.make_table(tspec, tseed)
        m = max(1, min(n_s, int(rate * per_step)))
        rec = gen.make_records(rspec, rseed, net, ln, n=m)
        t = time.perf_counter()
        o.discriminate_histogram(net, ln, rec, t0, w, nb)
        dt = time.perf_counter() - t
        if s >= args.warmup:
            done += m
            total += dt
    value = done / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": name, "records_per_step": done // args.steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.threads(), "kind": "oracle",
                             "sample": "a prefix of one slice (request) per step, taken in order"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_oracle_check(server, specs, pools, phase, args, tenant=None, k_random=2000, k_hot=200):
    """Compare a tenant's resident histogram with the oracle.

    Every request of a tenant covered the first n records of the tenant's
    pool, so record i was added as many times as there were requests longer
    than i: the expected histogram is, over the segments between consecutive
    request lengths, the segment's histogram times the number of requests
    that covered it (counts modulo 2^32, byte sums modulo 2^64). The oracle
    computes each segment on a sample of bins: random bins, the day's edges
    and the resident histogram's hottest bins."""
    import oracle

    o_ = oracle.get()
    done = phase[0][:max(3, args.warmup)] + phase[0] + phase[1] + phase[2]
    if tenant is None:  # the tenant with the most records submitted
        tot = {}
        for r in done:
            tot[r.tenant] = tot.get(r.tenant, 0) + r.n
        tenant = max(tot, key=tot.get)
    lens = sorted(r.n for r in done if r.tenant == tenant)
    got = server.export(tenant)
    nb = got["count"].shape[1]
    rng = np.random.default_rng(tenant)
    hot = np.argsort(got["count"][0].astype(np.uint64) + got["count"][1])[::-1][:k_hot]
    keep = np.unique(np.concatenate([rng.integers(0, nb, k_random), hot, [0, nb - 1]])).astype(np.uint64)
    net, ln = gen.make_table(specs[tenant], gen.BASE_SEED + 5000 + tenant)
    pool = pools[tenant]
    rec = {"ts": pool["ts"].numpy().view(np.uint64), "src": pool["src"].numpy().view(np.uint32),
           "dst": pool["dst"].numpy().view(np.uint32), "bytes": pool["bytes"].numpy().view(np.uint32)}
    want_c = np.zeros((2, len(keep)), np.uint64)
    want_b = np.zeros((2, len(keep)), np.uint64)
    t0 = time.perf_counter()
    lo = 0
    for j, hi in enumerate(lens):
        if hi > lo:
            seg = {k: v[lo:hi] for k, v in rec.items()}
            c, b = o_.histogram_bins(net, ln, seg, 0, 1, nb, keep)
            mult = np.uint64(len(lens) - j)
            with np.errstate(over="ignore"):
                want_c += c.astype(np.uint64) * mult
                want_b += b * mult
        lo = hi
    idx = keep.astype(np.int64)
    ok_c = np.array_equal((want_c & np.uint64(0xFFFFFFFF)).astype(np.uint32), got["count"][:, idx])
    ok_b = np.array_equal(want_b, got["bytes"][:, idx])
    ok_n = int(got["stats"][:4].sum()) == sum(lens)
    assert ok_c and ok_b and ok_n, f"serving tenant {tenant} differs from the oracle"
    return {"tenant": tenant, "requests": len(lens), "records_submitted": int(sum(lens)),
            "bins_compared": int(len(keep)), "hottest_compared": int(k_hot), "bit_exact": True,
            "oracle_s": round(time.perf_counter() - t0, 1)}


def run_serve_bench(args):
    """The serving loop: tenants with resident day histograms; request sizes
    log-normal (median 1 M records, p99 50 M before the cap), each uniform over
    a random window of its tenant's day. Saturated throughput first (all
    requests queued at once), then Poisson arrivals at 50% and 80% of it."""
    from dataclasses import replace

    rank, world, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    import paper_2106_12863_gb300 as sinet

    sinet.load()
    specs, reqs = gen.serving_plan(n_tenants=args.tenants, n_requests=3 * args.requests,
                                   seed=rank_seed(gen.BASE_SEED + 5, rank, 1000), cap=args.request_cap)
    tg = time.perf_counter()
    tables, pools = [], []
    cap = max(r.n for r in reqs)
    for i, sp in enumerate(specs):
        net, ln = gen.make_table(sp, gen.BASE_SEED + 5000 + i)
        tables.append(sinet.PrefixTable(net, ln))
    # one pinned pool of records per tenant; a request of n records for
    # tenant t is the first n records of a window-shaped stream of t's pool
    for i, sp in enumerate(specs):
        net, ln = gen.make_table(sp, gen.BASE_SEED + 5000 + i)
        n_i = max([r.n for r in reqs if r.tenant == i] + [1])
        pool = {"ts": torch.empty(n_i, dtype=torch.int64, pin_memory=True),
                "src": torch.empty(n_i, dtype=torch.int32, pin_memory=True),
                "dst": torch.empty(n_i, dtype=torch.int32, pin_memory=True),
                "bytes": torch.empty(n_i, dtype=torch.int32, pin_memory=True)}
        first = next((r for r in reqs if r.tenant == i), None)
        rs = first.records if first else gen.RecordSpec(n_i)
        gen.fill_records(replace(rs, n=n_i), gen.BASE_SEED + 6000 + i, net, ln, 0, n_i,
                         pool["ts"], pool["src"], pool["dst"], pool["bytes"])
        pools.append(pool)
    t_gen = time.perf_counter() - tg
    params = [sinet.HistParams(0, 1, gen.DAY_MS, accumulate=True) for _ in specs]
    server = sinet.Server(list(zip(tables, params)), budget_bytes=int(args.budget_gb * (1 << 30)),
                          max_requests_per_launch=256)

    def submit(r):
        p = pools[r.tenant]
        return server.submit(r.tenant, p["ts"][:r.n], p["src"][:r.n], p["dst"][:r.n], p["bytes"][:r.n])

    phase = [reqs[k * args.requests:(k + 1) * args.requests] for k in range(3)]
    # warm-up
    for k in [submit(r) for r in phase[0][:max(3, args.warmup)]]:
        server.wait(k)
    server.drain()
    server.stats(reset=True)
    # saturated: everything queued at once
    clocks = ClockSampler(local)
    time.sleep(0.3)
    clocks.mark(True)
    t0 = time.perf_counter()
    ks = [submit(r) for r in phase[0]]
    server.drain()
    t_sat = time.perf_counter() - t0
    clocks.mark(False)
    clk = clocks.stop()
    for k in ks:
        server.wait(k)
    st = server.stats(reset=True)
    n_sat = sum(r.n for r in phase[0])
    sat = n_sat / t_sat
    serving = {"saturated": {"records_per_s": sat, "requests": len(phase[0]), "launches": st["launches"],
                             "p50_ms": st["p50_latency_ns"] / 1e6, "p99_ms": st["p99_latency_ns"] / 1e6,
                             "gpu_busy_frac": st["busy_ns"] / 1e9 / t_sat}}
    mean_n = n_sat / len(phase[0])
    for rho, ph in ((0.5, phase[1]), (0.8, phase[2])):
        lam = rho * sat / mean_n  # requests per second
        ks, t_next = [], time.perf_counter()
        t_start = t_next
        for r in ph:
            t_next += r.gap / lam
            while time.perf_counter() < t_next:
                pass
            ks.append(submit(r))
        server.drain()
        t_el = time.perf_counter() - t_start
        for k in ks:
            server.wait(k)
        st = server.stats(reset=True)
        serving[f"rho_{rho}"] = {"offered_records_per_s": rho * sat,
                                 "achieved_records_per_s": sum(r.n for r in ph) / t_el,
                                 "requests": len(ph), "launches": st["launches"],
                                 "p50_ms": st["p50_latency_ns"] / 1e6, "p99_ms": st["p99_latency_ns"] / 1e6,
                                 "max_ms": st["max_latency_ns"] / 1e6}
    # full-scale parity: one tenant's resident day histogram, after every
    # phase, against the oracle over that tenant's requests (sampled bins)
    serving["oracle_check"] = serve_oracle_check(server, specs, pools, phase, args)
    h2d = RECORD_BYTES * mean_n
    result = {"metric": METRIC, "value": world * sat, "unit": UNIT, "n_gpus": world,
              "steps": len(phase[0]), "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t_sat / len(phase[0]),
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
              "data": "synthetic (seeded generator; Poisson request stream)"}
    peak, peak_kind = peaks()
    achieved = RECORD_BYTES * sat / 1e9
    result["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                          "frac": achieved / peak, "traffic": None, "kernel": "k_batch (serving launches)",
                          "peak_kind": peak_kind,
                          "note": "record bytes only, end to end: every record also crosses host-to-device"}
    result["gpu_launches"] = serving["saturated"]["launches"]
    result["e2e"] = {"value": world * sat, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                     "d2h_bytes_per_step": 0, "step": "one request (results stay resident)"}
    result["config"] = {"workload": f"serve-{len(specs)}-tenants-lognormal-1M", "tenants": len(specs),
                        "n_bins_per_tenant": gen.DAY_MS, "resident_gb": 24 * gen.DAY_MS * len(specs) / 1e9,
                        "inflight_budget_gb": args.budget_gb, "request_cap": args.request_cap,
                        "mean_request_records": mean_n, "policy": "exclusive",
                        "parallelism": f"replicas x{world} (weak)", "gen_s": round(t_gen, 1),
                        "l2": "inputs larger than L2"}
    result["serving"] = serving
    result["clocks"] = clk
    if rank == 0 and not args.no_cpu:
        import oracle

        o_ = oracle.get()
        done, t_cpu, i = 0, 0.0, 0
        while t_cpu < args.cpu_seconds and i < len(phase[0]):
            r = phase[0][i]
            net, ln = gen.make_table(specs[r.tenant], gen.BASE_SEED + 5000 + r.tenant)
            m = min(r.n, 2_000_000)
            p = pools[r.tenant]
            rec = {"ts": p["ts"][:m].numpy().view(np.uint64), "src": p["src"][:m].numpy().view(np.uint32),
                   "dst": p["dst"][:m].numpy().view(np.uint32), "bytes": p["bytes"][:m].numpy().view(np.uint32)}
            t0_ = time.perf_counter()
            o_.discriminate_histogram(net, ln, rec, 0, 1, gen.DAY_MS)
            t_cpu += time.perf_counter() - t0_
            done += m
            i += 1
        result["cpu_baseline"] = {"value": done / t_cpu, "unit": UNIT, "cores": o_.threads(), "kind": "oracle",
                                  "sample": f"{i} requests (at most 2 M records each, {done} records), "
                                            f"one oracle call each into a day histogram; {t_cpu:.1f} s"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    server.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch_bench(args)
        return
    if args.workload == "serve":
        run_serve_bench(args)
        return
    rank, world, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    import paper_2106_12863_gb300 as sinet

    sinet.load()  # fails loudly without the CUDA library

    w = workload(args, rank)
    result = run_window_bench(args, w, rank, world, dev, extras=True)
    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    # the paper-shaped time-sorted day as a second, smaller line of figures
    if args.workload == "heavy" and not args.no_day and not args.records and args.scale == 1.0:
        torch.cuda.empty_cache()
        day = run_window_bench(args, workload_named("day"), rank, world, dev, extras=False)
        result["day"] = {k: day[k] for k in ("value", "unit", "ms_per_step", "roofline", "config",
                                              "plain_sort_reduce", "fused_vs_plain", "clocks") if k in day}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_window_bench(args, w, rank, world, dev, extras: bool):
    """One window workload (tiny, day or heavy): tune, time K steps, the plain
    path, and (with extras) the end-to-end pipeline and the post-processing."""
    import torch

    import paper_2106_12863_gb300 as sinet

    from paper_2106_12863_gb300 import shard

    mode = args.shard if world > 1 else "single"
    n_total = w.records.n
    net, ln = gen.make_table(w.table, w.seed)
    tg = time.perf_counter()
    if mode == "time":
        # this rank owns bins [lo, hi) and is given the records that fall there
        if w.records.ts_kind != "diurnal":
            raise SystemExit("--shard time needs a time-sorted workload (day)")
        h, seed = owned_records(w, net, ln, world, rank), w.seed
        win = shard.Window(w.t0, w.bin_width, w.n_bins).owned(world, rank)
        n = int(h["ts"].numel())
    else:
        if mode == "records":  # this rank's share of one workload
            first, last = shard.record_range(n_total, world, rank)
            seed = w.seed
        else:  # replicas: every rank processes its own day (weak scaling)
            first, last = 0, n_total
            seed = rank_seed(w.seed, rank)
        n = last - first
        # records generated straight into pinned host memory, then made resident
        h = {"ts": torch.empty(n, dtype=torch.int64, pin_memory=True),
             "src": torch.empty(n, dtype=torch.int32, pin_memory=True),
             "dst": torch.empty(n, dtype=torch.int32, pin_memory=True),
             "bytes": torch.empty(n, dtype=torch.int32, pin_memory=True)}
        gen.fill_records(w.records, seed, net, ln, first, n, h["ts"], h["src"], h["dst"], h["bytes"])
        win = shard.Window(w.t0, w.bin_width, w.n_bins)
    t_gen = time.perf_counter() - tg
    d = {k: v.to(dev) for k, v in h.items()}
    table = sinet.PrefixTable(net, ln)
    out = sinet.Histogram(win.n_bins, dev, zero=False)
    stream = torch.cuda.current_stream(dev)
    hints = sinet.HINT_TIME_SORTED if w.records.ts_kind == "diurnal" else 0

    def params(strategy, accumulate=True):
        return sinet.HistParams(win.t0, win.width, win.n_bins, strategy=strategy, hints=hints,
                                accumulate=accumulate)

    def zero():
        out.count.zero_()
        out.bytes.zero_()
        out.stats.zero_()

    def writes_every_bin(strategy):
        # the cell strategy expands every bin into the outputs itself; the
        # owners and the partition's cold pass store every bin
        return strategy in ("atomic_cell", "owner", "partition")

    def step(strategy):
        if writes_every_bin(strategy):
            sinet.discriminate_histogram(table, d["ts"], d["src"], d["dst"], d["bytes"],
                                         params(strategy, accumulate=False), out)
            return
        zero()
        sinet.discriminate_histogram(table, d["ts"], d["src"], d["dst"], d["bytes"],
                                     params(strategy), out)

    # autotune: one untimed run of each candidate, keep the fastest. The
    # owner-computes scheme and the tile are for time-sorted input; unsorted
    # input over a histogram far beyond L2 leaves the partition, the cells
    # and the combining atomics (plain atomics there take ~10x longer)
    if args.strategy != "tune":
        cands = [args.strategy]
    elif hints:
        cands = ["owner", "priv_tile", "global_atomic", "atomic_cell", "partition"]
    else:
        cands = ["partition", "atomic_cell", "global_atomic"]
    tune = {}
    for c in cands:
        step(c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(c)
        e1.record(stream)
        torch.cuda.synchronize()
        tune[c] = e0.elapsed_time(e1)
    strategy = min(tune, key=tune.get)

    for _ in range(args.warmup):
        step(strategy)
    torch.cuda.synchronize()
    # timed region: K steps, zero + fused kernel, events on the launching stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(dev.index)
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.mark(True)
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_begin.record(stream)
    own = writes_every_bin(strategy)
    for i in range(args.steps):
        a, b, c = ev[i]
        a.record(stream)
        if not own:
            zero()
        b.record(stream)
        sinet.discriminate_histogram(table, d["ts"], d["src"], d["dst"], d["bytes"],
                                     params(strategy, accumulate=not own), out)
        if mode == "records":  # merge the ranks' partial histograms (each keeps its bin slice)
            shard.merge(out.count, out.bytes, out.stats, scatter=True)
        c.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks.mark(False)
    clk = clocks.stop()
    total_ms = t_begin.elapsed_time(t_end)
    kern_ms = statistics.mean(b.elapsed_time(c) for _, b, c in ev)
    zero_ms = statistics.mean(a.elapsed_time(b) for a, b, _ in ev)
    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / args.steps
    if mode in ("records", "time"):  # one workload over all ranks (strong scaling)
        value = n_total * args.steps / (total_ms / 1e3)
    else:
        value = job_rate(n, world, args.steps, total_ms)
    stats = out.stats.cpu().numpy().view(np.uint64)
    # invariant spot check on the last step: every record classified once
    # (after a record-range merge the counters hold every rank's records)
    assert int(stats[:4].sum()) == (n_total if mode == "records" else n), \
        "class counts do not sum to the record count"

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
              "scaling": "strong" if mode in ("records", "time") else "weak", "vs_baseline": None,
              "dtype": "u32/u64", "data": f"synthetic (seeded generator; {w.name})"}
    alg_bytes = RECORD_BYTES * n + BIN_BYTES * win.n_bins
    peak, peak_kind = peaks()
    kname = {"owner": "k_fused_owner", "priv_tile": "k_fused_tile", "global_atomic": "k_fused_atomic",
             "atomic_noagg": "k_fused_atomic", "atomic_cell": "k_fused_atomic",
             "partition": "k_part_main", "sort_reduce": "k_radix_pass"}[strategy]
    # the fraction counts everything a step needs (the zeroing that the tile
    # and atomic schemes require included): algorithmic bytes over the step
    achieved = alg_bytes / (ms_per_step / 1e3) / 1e9
    result["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                          "frac": achieved / peak, "traffic": recorded_traffic(kname, w.name),
                          "kernel": kname, "peak_kind": peak_kind,
                          "algorithmic_bytes_per_launch": alg_bytes,
                          "step_ms": ms_per_step, "call_ms": kern_ms, "zero_ms": zero_ms,
                          "call_frac": alg_bytes / (kern_ms / 1e3) / 1e9 / peak,
                          "timed": "whole step (CUDA events on the launching stream): "
                                   + ("the library call" if own else "output zeroing + the library call")}
    # kernels per step: one fused kernel (zeroing is cudaMemsetAsync), plus
    # the cell expansion for the cell strategy; the run boundaries, their scan
    # and the remainder for the owner strategy; sample, levels, total,
    # candidates, hot table, main pass, three page-grouping kernels, cold pass
    # and hot totals for the partition
    result["gpu_launches"] = args.steps * {"atomic_cell": 2, "owner": 4, "partition": 11}.get(strategy, 1)
    result["config"] = {"workload": w.name, "records": n, "prefixes": w.table.n,
                        "n_bins": w.n_bins, "bin_width_ms": w.bin_width, "strategy": strategy,
                        "tune_ms": tune, "l2": f"inputs larger than L2 ({RECORD_BYTES * n / 1e9:.1f} GB of records)",
                        "policy": "exclusive", "parallelism": {
                            "single": "1 GPU", "replicas": f"replicas x{world} (weak)",
                            "records": f"record-range split x{world} + NCCL reduce-scatter of the "
                                       "histogram in every step (strong)",
                            "time": f"owned bin ranges x{world}, no collective (strong)"}[mode],
                        "records_this_rank": n,
                        "gen_s": round(t_gen, 1), "seed": seed,
                        "data_sha256_prefix": data_digest([h["ts"], h["src"], h["dst"], h["bytes"]])}
    result["clocks"] = clk

    # the plain path (paper's structure) on the same data
    if not args.no_plain:
        for _ in range(2):
            step("sort_reduce")
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.plain_steps):
            step("sort_reduce")
        p1.record(stream)
        torch.cuda.synchronize()
        plain_ms = p0.elapsed_time(p1) / args.plain_steps
        result["plain_sort_reduce"] = {"value": n / (plain_ms / 1e3), "unit": UNIT,
                                       "ms_per_step": plain_ms, "steps": args.plain_steps}
        result["fused_vs_plain"] = (n / (ms_per_step / 1e3)) / result["plain_sort_reduce"]["value"]

    # end to end through the public API: pinned host records in, histogram out.
    # Two buffer sets on two streams: the host link carries one direction at
    # a time per stream, so step k's histogram read-back overlaps step k+1's
    # record upload (the steady state of a stream of days).
    if extras and not args.no_e2e:
        nbuf = 2
        dsets = [d] + [{k: torch.empty_like(v) for k, v in d.items()} for _ in range(nbuf - 1)]
        outs = [out] + [sinet.Histogram(win.n_bins, dev, zero=False) for _ in range(nbuf - 1)]
        houts = [{"count": torch.empty((2, win.n_bins), dtype=torch.int32, pin_memory=True),
                  "bytes": torch.empty((2, win.n_bins), dtype=torch.int64, pin_memory=True),
                  "stats": torch.empty(8, dtype=torch.int64, pin_memory=True)} for _ in range(nbuf)]
        e2e_streams = [torch.cuda.Stream(dev) for _ in range(nbuf)]

        def e2e_step(k):
            i = k % nbuf
            s_ = e2e_streams[i]
            with torch.cuda.stream(s_):
                for key in d:
                    dsets[i][key].copy_(h[key], non_blocking=True)
                sinet.discriminate_histogram(table, dsets[i]["ts"], dsets[i]["src"], dsets[i]["dst"],
                                             dsets[i]["bytes"], params(strategy, accumulate=False),
                                             outs[i], stream=s_)
                houts[i]["count"].copy_(outs[i].count, non_blocking=True)
                houts[i]["bytes"].copy_(outs[i].bytes, non_blocking=True)
                houts[i]["stats"].copy_(outs[i].stats, non_blocking=True)

        for k in range(nbuf):
            e2e_step(k)
        torch.cuda.synchronize()
        t_e = time.perf_counter()
        for k in range(args.e2e_steps):
            e2e_step(k)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t_e) * 1e3 / args.e2e_steps
        h2d = sum(v.numel() * v.element_size() for v in h.values())
        d2h = sum(v.numel() * v.element_size() for v in houts[0].values())
        result["e2e"] = {"value": world * n / (e2e_ms / 1e3), "unit": UNIT,
                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                         "ms_per_step": e2e_ms, "steps": args.e2e_steps,
                         "pipelining": "2 buffer sets on 2 streams; host wall clock"}
        for ho in houts:
            st2 = ho["stats"].numpy().view(np.uint64)
            assert np.array_equal(st2, stats), "e2e result differs from the resident run"
        del dsets[1:], outs[1:]

    # post-processing of the day histogram: hourly and ten-minute roll-ups and
    # the sparse form (each reads the 24 B per bin of the dense histogram)
    if extras and not args.no_post and w.bin_width == 1:
        post = {}
        hist_bytes = BIN_BYTES * win.n_bins
        for name, fn in (("rollup_10min", lambda: sinet.rollup(out, 600_000, out=coarse10)),
                         ("rollup_1h", lambda: sinet.rollup(out, 3_600_000, out=coarse1h)),
                         ("sparse", lambda: sinet.sinet_histogram_sparse(
                             out.c(), win.n_bins, sp_bin, sp_c[0], sp_c[1], sp_b[0], sp_b[1], win.n_bins, sp_n))):
            if name == "rollup_10min":
                coarse10 = sinet.Histogram(-(-win.n_bins // 600_000), dev, zero=False)
                coarse1h = sinet.Histogram(-(-win.n_bins // 3_600_000), dev, zero=False)
                sp_bin = torch.empty(win.n_bins, dtype=torch.int32, device=dev)
                sp_c = torch.empty((2, win.n_bins), dtype=torch.int32, device=dev)
                sp_b = torch.empty((2, win.n_bins), dtype=torch.int64, device=dev)
                sp_n = torch.zeros(1, dtype=torch.int64, device=dev)
            fn()
            torch.cuda.synchronize()
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            for _ in range(5):
                fn()
            p1.record(stream)
            torch.cuda.synchronize()
            ms = p0.elapsed_time(p1) / 5
            post[name] = {"ms": ms, "input_GBs": hist_bytes / (ms / 1e3) / 1e9}
        post["sparse"]["bins"] = int(sp_n.item())
        # a watch list of 877 hosts (the size of the paper's larger blocklist),
        # drawn from the day's own addresses so that some sessions match
        rng = np.random.default_rng(877)
        hs = h["src"][: 1 << 20].numpy().view(np.uint32)
        wnet = np.unique(rng.choice(hs, 877)).astype(np.uint32)
        watch = sinet.PrefixTable(wnet, np.full(len(wnet), 32, np.uint8))
        wp = sinet.HistParams(win.t0, win.width, win.n_bins, watch=watch)

        def watched():
            sinet.discriminate_histogram(table, d["ts"], d["src"], d["dst"], d["bytes"], wp, out)

        watched()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(5):
            watched()
        p1.record(stream)
        torch.cuda.synchronize()
        ms = p0.elapsed_time(p1) / 5
        kept = n - int(out.stats.cpu().numpy().view(np.uint64)[6])
        post["watch_877_hosts"] = {"ms": ms, "sessions_per_s": n / (ms / 1e3), "kept": kept}
        watch.close()

        # the split entry points: Algorithm 1 alone (class bytes out), then the
        # histogram of those classes (8 + 1 and 12 + 1 bytes per record read)
        cls = torch.empty(n, dtype=torch.uint8, device=dev)
        hp = sinet.HistParams(win.t0, win.width, win.n_bins, strategy="priv_tile" if hints else "atomic_cell",
                              hints=hints)
        for name, fn, per_rec in (
                ("discriminate", lambda: sinet.discriminate(table, d["src"], d["dst"], cls), 9),
                ("histogram_from_classes", lambda: sinet.histogram(d["ts"], d["bytes"], cls, hp, out), 13)):
            fn()
            torch.cuda.synchronize()
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            for _ in range(5):
                fn()
            p1.record(stream)
            torch.cuda.synchronize()
            ms = p0.elapsed_time(p1) / 5
            extra = BIN_BYTES * win.n_bins if name == "histogram_from_classes" else 0
            post[name] = {"ms": ms, "sessions_per_s": n / (ms / 1e3),
                          "algorithmic_GBs": (per_rec * n + extra) / (ms / 1e3) / 1e9}
        del cls
        result["post"] = post
        del sp_bin, sp_c, sp_b

    table.close()
    return result


if __name__ == "__main__":
    main()
