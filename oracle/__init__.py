"""Plain CPU oracle for the session-discrimination hot path.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package. It shares no code with the
CUDA library (``paper_2106_12863_gb300``) and never imports it.

The arithmetic lives in ``sinet_oracle.c`` (Algorithm 1 per record and per
CIDR entry; the millisecond histogram of Section 5); this module only marshals
numpy arrays. Policies map a class (0 neither, 1 src inside, 2 dst inside,
3 both) to a direction set (bit 0 outgoing, bit 1 ingoing).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "sinet_oracle.c")
LIB_PATH = os.path.join(_HERE, "_lib", "liboracle.so")

#: class -> direction set; EXCLUSIVE bins only one-sided sessions
EXCLUSIVE = (0, 1, 2, 0)
#: the literal Algorithm 1: source inside -> outgoing, otherwise ingoing
PAPER_ALG1 = (2, 1, 2, 1)
#: sessions with both ends inside count in both directions
INCLUSIVE = (0, 1, 2, 3)


def _bind(L):
    P = ctypes.c_void_p
    u64 = ctypes.c_uint64
    L.oracle_bitmask.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
    L.oracle_bitmask.restype = ctypes.c_uint32
    L.oracle_in_list.argtypes = [ctypes.c_uint32, P, P, ctypes.c_uint32]
    L.oracle_in_list.restype = ctypes.c_int
    L.oracle_classify.argtypes = [P, P, ctypes.c_uint32, P, P, u64, P]
    L.oracle_classify.restype = None
    L.oracle_histogram.argtypes = [P, P, P, u64, u64, u64, u64, P, P, P, P, P, P]
    L.oracle_histogram.restype = None
    L.oracle_discriminate_histogram.argtypes = [P, P, ctypes.c_uint32, P, P, P, P, u64, u64, u64,
                                                u64, P, P, P, P, P, P]
    L.oracle_discriminate_histogram.restype = ctypes.c_int
    L.oracle_discriminate_histogram_watch.argtypes = [P, P, ctypes.c_uint32, P, P, ctypes.c_uint32, P, P, P,
                                                      P, u64, u64, u64, u64, P, P, P, P, P, P]
    L.oracle_discriminate_histogram_watch.restype = ctypes.c_int
    L.oracle_histogram_bins.argtypes = [P, P, ctypes.c_uint32, P, P, P, P, u64, u64, u64, u64, P,
                                        P, u64, P, P]
    L.oracle_histogram_bins.restype = None
    L.oracle_num_threads.restype = ctypes.c_int
    L.oracle_mutant.restype = ctypes.c_int
    return L


class Oracle:
    """One loaded build of the oracle (the default, or a planted-mistake build)."""

    def __init__(self, path: str = LIB_PATH):
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run __graft_entry__.build() first")
        self.L = _bind(ctypes.CDLL(path))
        self.path = path

    # -- Algorithm 1 -----------------------------------------------------
    def bitmask(self, x: int, z: int) -> int:
        return int(self.L.oracle_bitmask(x, z))

    def in_list(self, x: int, net, ln) -> bool:
        net = np.ascontiguousarray(net, np.uint32)
        ln = np.ascontiguousarray(ln, np.uint8)
        return bool(self.L.oracle_in_list(x, net.ctypes.data, ln.ctypes.data, len(net)))

    def classify(self, net, ln, src, dst) -> np.ndarray:
        net = np.ascontiguousarray(net, np.uint32)
        ln = np.ascontiguousarray(ln, np.uint8)
        src = np.ascontiguousarray(src, np.uint32)
        dst = np.ascontiguousarray(dst, np.uint32)
        out = np.empty(len(src), np.uint8)
        self.L.oracle_classify(net.ctypes.data, ln.ctypes.data, len(net), src.ctypes.data,
                               dst.ctypes.data, len(src), out.ctypes.data)
        return out

    # -- histogram ----------------------------------------------------------
    @staticmethod
    def empty_hist(n_bins: int):
        return {
            "count": np.zeros((2, n_bins), np.uint32),
            "bytes": np.zeros((2, n_bins), np.uint64),
            "stats": np.zeros(8, np.uint64),
        }

    def histogram(self, ts, nbytes, cls, t0, w, n_bins, policy=EXCLUSIVE, into=None):
        h = self.empty_hist(n_bins) if into is None else into
        ts = np.ascontiguousarray(ts, np.uint64)
        nbytes = np.ascontiguousarray(nbytes, np.uint32)
        cls = np.ascontiguousarray(cls, np.uint8)
        pol = np.asarray(policy, np.uint8)
        c, b, s = h["count"], h["bytes"], h["stats"]
        self.L.oracle_histogram(ts.ctypes.data, nbytes.ctypes.data, cls.ctypes.data, len(ts), t0, w,
                                n_bins, pol.ctypes.data, c[0].ctypes.data, c[1].ctypes.data,
                                b[0].ctypes.data, b[1].ctypes.data, s.ctypes.data)
        return h

    def discriminate_histogram(self, net, ln, rec, t0, w, n_bins, policy=EXCLUSIVE, into=None):
        h = self.empty_hist(n_bins) if into is None else into
        net = np.ascontiguousarray(net, np.uint32)
        ln = np.ascontiguousarray(ln, np.uint8)
        ts = np.ascontiguousarray(rec["ts"], np.uint64)
        src = np.ascontiguousarray(rec["src"], np.uint32)
        dst = np.ascontiguousarray(rec["dst"], np.uint32)
        nb = np.ascontiguousarray(rec["bytes"], np.uint32)
        pol = np.asarray(policy, np.uint8)
        c, b, s = h["count"], h["bytes"], h["stats"]
        rc = self.L.oracle_discriminate_histogram(
            net.ctypes.data, ln.ctypes.data, len(net), ts.ctypes.data, src.ctypes.data,
            dst.ctypes.data, nb.ctypes.data, len(ts), t0, w, n_bins, pol.ctypes.data,
            c[0].ctypes.data, c[1].ctypes.data, b[0].ctypes.data, b[1].ctypes.data, s.ctypes.data)
        if rc != 0:
            raise MemoryError("oracle allocation failed")
        return h

    def discriminate_histogram_watch(self, net, ln, wnet, wln, rec, t0, w, n_bins, policy=EXCLUSIVE,
                                     into=None):
        """Only records with src or dst in the watch list (wnet, wln) are classified and binned;
        the others count in stats[6]."""
        h = self.empty_hist(n_bins) if into is None else into
        net = np.ascontiguousarray(net, np.uint32)
        ln = np.ascontiguousarray(ln, np.uint8)
        wnet = np.ascontiguousarray(wnet, np.uint32)
        wln = np.ascontiguousarray(wln, np.uint8)
        ts = np.ascontiguousarray(rec["ts"], np.uint64)
        src = np.ascontiguousarray(rec["src"], np.uint32)
        dst = np.ascontiguousarray(rec["dst"], np.uint32)
        nb = np.ascontiguousarray(rec["bytes"], np.uint32)
        pol = np.asarray(policy, np.uint8)
        c, b, s = h["count"], h["bytes"], h["stats"]
        rc = self.L.oracle_discriminate_histogram_watch(
            net.ctypes.data, ln.ctypes.data, len(net), wnet.ctypes.data if len(wnet) else None,
            wln.ctypes.data if len(wln) else None, len(wnet), ts.ctypes.data, src.ctypes.data,
            dst.ctypes.data, nb.ctypes.data, len(ts), t0, w, n_bins, pol.ctypes.data,
            c[0].ctypes.data, c[1].ctypes.data, b[0].ctypes.data, b[1].ctypes.data, s.ctypes.data)
        if rc != 0:
            raise MemoryError("oracle allocation failed")
        return h

    def histogram_bins(self, net, ln, rec, t0, w, n_bins, keep, policy=EXCLUSIVE):
        """Full-workload values of the sorted bins ``keep``: (count[2, m], bytes[2, m])."""
        net = np.ascontiguousarray(net, np.uint32)
        ln = np.ascontiguousarray(ln, np.uint8)
        keep = np.ascontiguousarray(keep, np.uint64)
        assert np.all(keep[1:] > keep[:-1])
        m = len(keep)
        cnt = np.zeros(2 * m, np.uint32)
        byt = np.zeros(2 * m, np.uint64)
        ts = np.ascontiguousarray(rec["ts"], np.uint64)
        src = np.ascontiguousarray(rec["src"], np.uint32)
        dst = np.ascontiguousarray(rec["dst"], np.uint32)
        nb = np.ascontiguousarray(rec["bytes"], np.uint32)
        pol = np.asarray(policy, np.uint8)
        self.L.oracle_histogram_bins(net.ctypes.data, ln.ctypes.data, len(net), ts.ctypes.data,
                                     src.ctypes.data, dst.ctypes.data, nb.ctypes.data, len(ts), t0,
                                     w, n_bins, pol.ctypes.data, keep.ctypes.data, m,
                                     cnt.ctypes.data, byt.ctypes.data)
        return cnt.reshape(2, m), byt.reshape(2, m)

    def threads(self) -> int:
        return int(self.L.oracle_num_threads())

    def mutant(self) -> int:
        return int(self.L.oracle_mutant())


_default = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def compile_variant(out_path: str, mutant: int = 0, openmp: bool = True) -> str:
    """Compile the oracle source (optionally with a planted mistake) to ``out_path``."""
    import subprocess

    cmd = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", f"-DORACLE_MUTANT={mutant}", SOURCE,
           "-o", out_path]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    return out_path
