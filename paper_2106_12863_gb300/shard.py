"""One workload split across ranks (one process per GPU), after the paper's
multi-GPU setting: each GPU takes its own chunk of the records and the
per-GPU partial histograms are merged (Section 5's pairwise reduction and
merge scatter; Table 3's four-GPU runs).

Two splits, both exact (the histogram is an integer sum):

- by record range: rank r discriminates and histograms records
  [lo_r, hi_r) into full-size partial histograms, which a sum-reduction over
  ranks merges. Counts (uint32, modulo 2^32) and byte sums (uint64, modulo
  2^64) travel as separate collectives, bit for bit as int32 / int64, whose
  two's-complement sums wrap exactly as the unsigned ones do. ``merge``
  either gives every rank the whole result (all-reduce) or leaves rank r the
  bins [bin_lo_r, bin_hi_r) of it (reduce-scatter), the latter moving
  (world - 1) / world of the histogram per rank instead of twice that.
- by time range: rank r owns the bins [bin_lo_r, bin_hi_r) and is given the
  records whose bin falls there (for time-sorted input, a contiguous run of
  records); its histogram of that window is final, so no reduction is
  needed, and ``gather_owned`` assembles the whole histogram where wanted.

The per-rank compute is the library call (``discriminate_histogram``) on the
rank's own device; this module only splits ranges and moves results with
``torch.distributed`` (NCCL on GPUs, gloo on CPUs). It holds none of the
method's arithmetic beyond the integer sum of the merge.
"""
from __future__ import annotations

from dataclasses import dataclass


def record_range(n: int, world: int, rank: int, align: int = 4) -> tuple[int, int]:
    """Records [lo, hi) of rank ``rank``: near-equal shares whose boundaries
    are multiples of ``align`` (so every rank's streams keep the alignment of
    the whole arrays), the last rank taking the remainder."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    if align < 1:
        raise ValueError("align must be >= 1")
    units = -(-n // align)
    lo = min(n, (units * rank // world) * align)
    hi = min(n, (units * (rank + 1) // world) * align)
    return lo, hi


def bin_range(n_bins: int, world: int, rank: int) -> tuple[int, int]:
    """Bins [lo, hi) owned by ``rank`` under the time-range split (and the
    slice a reduce-scatter leaves on it): near-equal contiguous shares."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return n_bins * rank // world, n_bins * (rank + 1) // world


@dataclass(frozen=True)
class Window:
    """A histogram window: bins [0, n_bins) of width ``width`` from ``t0``."""
    t0: int
    width: int
    n_bins: int

    def owned(self, world: int, rank: int) -> "Window":
        """The sub-window of the bins ``rank`` owns (time-range split)."""
        lo, hi = bin_range(self.n_bins, world, rank)
        return Window(self.t0 + lo * self.width, self.width, max(hi - lo, 0))


def _flat_views(count, nbytes):
    """Bit-preserving int32 / int64 views of [2, n_bins] uint32 / uint64 arrays."""
    import torch

    c = count if count.dtype == torch.int32 else count.view(torch.int32)
    b = nbytes if nbytes.dtype == torch.int64 else nbytes.view(torch.int64)
    return c, b


def merge(count, nbytes, stats, group=None, scatter: bool = False):
    """Sum the ranks' partial histograms (record-range split).

    ``count`` [2, n_bins] int32 (uint32 bits), ``nbytes`` [2, n_bins] int64
    (uint64 bits), ``stats`` [8] int64 on this rank's device. With
    ``scatter`` False every rank ends with the whole sum in place; with True
    the sum of bins [bin_range(n_bins, world, rank)) is returned as new
    (count, nbytes) tensors [2, hi - lo] and the inputs are left as they were
    (stats are all-reduced in place either way)."""
    import torch
    import torch.distributed as dist

    c, b = _flat_views(count, nbytes)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dist.all_reduce(stats, op=dist.ReduceOp.SUM, group=group)
    if not scatter:
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(b, op=dist.ReduceOp.SUM, group=group)
        return count, nbytes
    n_bins = c.shape[1]
    bounds = [bin_range(n_bins, world, r) for r in range(world)]
    outs = []
    for x in (c, b):
        # one direction after the other keeps every rank's slice contiguous
        res = torch.empty((2, bounds[rank][1] - bounds[rank][0]), dtype=x.dtype, device=x.device)
        for dd in range(2):
            parts = [x[dd, lo:hi].contiguous() for lo, hi in bounds]
            if all(p.numel() == parts[0].numel() for p in parts) and dist.get_backend(group) != "gloo":
                dist.reduce_scatter(res[dd], parts, op=dist.ReduceOp.SUM, group=group)
            else:
                # unequal slices (or gloo, which has no reduce_scatter): a
                # reduce of each slice to its owner
                for r, (lo, hi) in enumerate(bounds):
                    buf = x[dd, lo:hi].contiguous()
                    dist.reduce(buf, dst=dist.get_global_rank(group, r) if group is not None else r,
                                op=dist.ReduceOp.SUM, group=group)
                    if r == rank:
                        res[dd].copy_(buf)
        outs.append(res)
    return outs[0], outs[1]


def gather_owned(count, nbytes, stats, n_bins: int, group=None):
    """Assemble the whole histogram on every rank from the ranks' owned
    slices (time-range split): ``count`` / ``nbytes`` are this rank's
    [2, hi - lo] slices. Stats are summed."""
    import torch
    import torch.distributed as dist

    c, b = _flat_views(count, nbytes)
    world = dist.get_world_size(group)
    bounds = [bin_range(n_bins, world, r) for r in range(world)]
    dist.all_reduce(stats, op=dist.ReduceOp.SUM, group=group)
    m = max(hi - lo for lo, hi in bounds)
    outs = []
    for x in (c, b):
        full = torch.empty((2, n_bins), dtype=x.dtype, device=x.device)
        for dd in range(2):
            # equal-size pieces (slices differ by at most one bin): pad, gather, trim
            mine = torch.zeros(m, dtype=x.dtype, device=x.device)
            mine[: x.shape[1]] = x[dd]
            parts = [torch.empty(m, dtype=x.dtype, device=x.device) for _ in bounds]
            dist.all_gather(parts, mine, group=group)
            for (lo, hi), p in zip(bounds, parts):
                full[dd, lo:hi] = p[: hi - lo]
        outs.append(full)
    return outs[0], outs[1]
