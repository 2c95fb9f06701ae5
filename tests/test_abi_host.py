"""Host-side checks of the C-ABI library (no GPU needed).

* the shared library loads and exports every function include/sinet.h declares;
* the CIDR parser agrees with Python's ``ipaddress``;
* the host table compiler (canonical groups, merged intervals, direct index)
  answers membership exactly like the oracle's per-entry loop;
* argument validation rejects bad input before any CUDA call.
"""
import ctypes
import ipaddress
import os
import random
import re

import numpy as np
import pytest

import gen
import paper_2106_12863_gb300 as sinet

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2106_12863_gb300 import _build

    _build.build()
    sinet.load()


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sinet_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    L = ctypes.CDLL(sinet.LIB_PATH)
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            names += _declared(h)
    assert "sinet_discriminate_histogram" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_header_compiles_as_c_and_cpp(tmp_path):
    """include/sinet.h is a plain C header: it compiles as C11 (pedantic) and C++17."""
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    src = tmp_path / "use.c"
    src.write_text('#include "sinet.h"\n'
                   "int main(void) { sinet_hist_params p; sinet_default_params(&p, 0, 1, 10);\n"
                   "  sinet_batch_slice b; sinet_server_config c; (void)b; (void)c;\n"
                   "  return (int)p.n_bins - 10; }\n")
    inc = os.path.join(ROOT, "include")
    for cmd in (["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only"],
                ["g++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-x", "c++"]):
        r = subprocess.run(cmd + ["-I", inc, str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_version_and_status_strings():
    assert sinet.sinet_version() >= 0x000100
    L = sinet.load()
    for code in range(9):
        assert L.sinet_status_string(code)
    assert L.sinet_status_string(99) == b"unknown status"


@pytest.mark.parametrize("text", ["192.168.1.5/24", "10.0.0.0/8", "0.0.0.0/0", "255.255.255.255/32",
                                  "1.2.3.4", "172.16.5.4/12"])
def test_parse_cidr_matches_ipaddress(text):
    net, ln = sinet.sinet_parse_cidr(text)
    iface = ipaddress.ip_interface(text)
    assert net == int(iface.ip)
    assert ln == iface.network.prefixlen


@pytest.mark.parametrize("bad", ["", "1.2.3", "1.2.3.4/33", "256.1.1.1/8", "1.2.3.4/", "a.b.c.d/8",
                                 "1.2.3.4/8x", "1..2.3/8", "1.2.3.4.5/8", "1234.1.1.1/8"])
def test_parse_cidr_rejects(bad):
    with pytest.raises(sinet.SinetError):
        sinet.sinet_parse_cidr(bad)


def _member_intervals(lo, hi, addrs):
    j = np.searchsorted(lo, addrs, side="right") - 1
    ok = j >= 0
    jj = np.where(ok, j, 0)
    return ok & (addrs <= hi[jj]) if len(lo) else np.zeros(len(addrs), bool)


def _member_index(lo, hi, index, k, addrs):
    """Membership through the direct index exactly as the kernels walk it."""
    out = np.zeros(len(addrs), bool)
    n = len(lo)
    for i, a in enumerate(addrs.tolist()):
        b = a >> (32 - k)
        j, e = int(index[b]), int(index[b + 1])
        if j >= n:
            continue
        e = min(e, n - 1)
        cand = [c for c in range(j, e + 1) if lo[c] <= a]
        if cand and a <= hi[cand[-1]]:
            out[i] = True
    return out


def _random_table(rng, k):
    net = np.array([rng.getrandbits(32) for _ in range(k)], np.uint32)  # host bits set on purpose
    ln = np.array([rng.choice([0, 1, 8, 9, 16, 20, 24, 25, 31, 32, rng.randint(0, 32)])
                   for _ in range(k)], np.uint8)
    return net, ln


def _edge_addrs(net, ln, rng, extra=400):
    a = [rng.getrandbits(32) for _ in range(extra)]
    for n, z in zip(net.tolist(), ln.tolist()):
        nw = ipaddress.ip_network((n, z), strict=False)
        lo, hi = int(nw.network_address), int(nw.broadcast_address)
        a += [lo, hi, (lo - 1) & 0xFFFFFFFF, (hi + 1) & 0xFFFFFFFF]
    return np.array(a, np.uint32)


@pytest.mark.parametrize("seed", range(8))
def test_compiled_table_equals_oracle(orc, seed):
    rng = random.Random(seed)
    net, ln = _random_table(rng, rng.randint(1, 40))
    addrs = _edge_addrs(net, ln, rng)
    want = orc.classify(net, ln, addrs, np.zeros_like(addrs)) & 1
    for k in (0, 6, 11):
        t = sinet.sinet_compile_prefix_table(net, ln, k)
        got = _member_intervals(t["lo"], t["hi"], addrs)
        assert np.array_equal(got, want.astype(bool))
        got2 = _member_index(t["lo"], t["hi"], t["index"], t["index_bits"], addrs)
        assert np.array_equal(got2, want.astype(bool))
        # intervals are sorted, disjoint and non-adjacent
        lo, hi = t["lo"].astype(np.int64), t["hi"].astype(np.int64)
        assert np.all(lo <= hi) and np.all(lo[1:] > hi[:-1] + 1)
        # canonical, deduplicated, grouped by length
        off = t["len_offset"]
        for L in range(33):
            g = t["nets"][off[L]:off[L + 1]]
            m = 0 if L == 0 else (0xFFFFFFFF << (32 - L)) & 0xFFFFFFFF
            assert np.all(g & np.uint32(m) == g)
            assert np.all(g[1:] > g[:-1])
        assert t["n_unique"] == len({(int(n) & ((0xFFFFFFFF << (32 - int(z))) & 0xFFFFFFFF if z else 0),
                                      int(z)) for n, z in zip(net, ln)})


def test_compiled_workload_tables(orc):
    rng = random.Random(3)
    for key in ("tiny", "day", "heavy"):
        w = gen.WORKLOADS[key]
        net, ln = gen.make_table(w.table, w.seed)
        t = sinet.sinet_compile_prefix_table(net, ln)
        assert t["max_range"] <= 4
        addrs = _edge_addrs(net[:300], ln[:300], rng, extra=3000)
        want = orc.classify(net, ln, addrs, np.zeros_like(addrs)) & 1
        assert np.array_equal(_member_intervals(t["lo"], t["hi"], addrs), want.astype(bool))


def test_empty_table_compiles():
    t = sinet.sinet_compile_prefix_table(np.zeros(0, np.uint32), np.zeros(0, np.uint8))
    assert t["n_unique"] == 0 and t["n_intervals"] == 0


def test_compile_rejects_bad_lengths():
    with pytest.raises(sinet.SinetError) as e:
        sinet.sinet_compile_prefix_table(np.array([1], np.uint32), np.array([33], np.uint8))
    assert e.value.status == 1
    with pytest.raises(sinet.SinetError):
        sinet.sinet_compile_prefix_table(np.array([1], np.uint32), np.array([8], np.uint8), 21)


def test_validation_rejects_before_any_cuda_call():
    """Bad parameters return SINET_ERR_INVALID_ARG without touching a device."""
    L = sinet.load()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    out = sinet.HistOutC()
    for i in range(2):
        out.count[i] = 0x10000
        out.bytes[i] = 0x20000
    out.stats = 0x30000
    for kw in ({"bin_width_ms": 0}, {"n_bins": 0}, {"n_bins": 1 << 31},
               {"t0_ms": (1 << 64) - 10, "n_bins": 100}):
        p = sinet.HistParams(t0_ms=kw.get("t0_ms", 0), bin_width_ms=kw.get("bin_width_ms", 1),
                             n_bins=kw.get("n_bins", 10)).c()
        rc = L.sinet_discriminate_histogram(fake, 0x40000, 0x50000, 0x60000, 0x70000, 8,
                                            ctypes.byref(p), ctypes.byref(out), None)
        assert rc == 1, kw
    p = sinet.HistParams(0, 1, 10, policy=(0, 1, 2, 4)).c()
    assert L.sinet_histogram(0x40000, 0x50000, 0x60000, 8, ctypes.byref(p), ctypes.byref(out), None) == 1
    p = sinet.HistParams(0, 1, 10).c()
    bad = sinet.HistOutC()
    assert L.sinet_histogram(0x40000, 0x50000, 0x60000, 8, ctypes.byref(p), ctypes.byref(bad), None) == 1
    # misaligned record pointer
    assert L.sinet_histogram(0x40004, 0x50000, 0x60000, 8, ctypes.byref(p), ctypes.byref(out), None) == 1
    assert L.sinet_discriminate(None, 0x40000, 0x50000, 8, None, 0x60000, 0, None) == 1


def test_batch_validation_rejects_before_any_cuda_call():
    """sinet_batch_create checks every slice on the host before touching a device."""
    L = sinet.load()
    h = ctypes.c_void_p()

    def good():
        c = sinet.BatchSliceC()
        c.ts, c.src, c.dst, c.bytes, c.n, c.table = 0x40000, 0x50000, 0x60000, 0x70000, 8, 0x1000
        c.params = sinet.HistParams(0, 1, 10).c()
        for i in range(2):
            c.out.count[i] = 0x10000
            c.out.bytes[i] = 0x20000
        c.out.stats = 0x30000
        return c

    def create(cs, flags=0):
        arr = (sinet.BatchSliceC * max(len(cs), 1))(*cs)
        return L.sinet_batch_create(arr if cs else None, len(cs), flags, None, ctypes.byref(h))

    assert create([]) == 1
    assert create([good()], flags=2) == 1
    bad = []
    c = good(); c.table = None; bad.append((c, 1))
    c = good(); c.params.bin_width_ms = 0; bad.append((c, 1))
    c = good(); c.ts = 0x40004; bad.append((c, 1))
    c = good(); c.out.stats = None; bad.append((c, 1))
    c = good(); c.params.strategy = sinet.STRAT_OWNER; bad.append((c, 8))
    c = good(); c.params.strategy = sinet.STRAT_PARTITION; bad.append((c, 8))
    c = good(); c.params.strategy = sinet.STRAT_PRIV_TILE; bad.append((c, 8))
    c = good(); c.params.lookup = sinet.LOOKUP_PML; bad.append((c, 8))
    for c, want in bad:
        assert create([good(), c]) == want
    assert L.sinet_batch_run(None, None) == 1
    assert L.sinet_batch_destroy(None) == 0


def test_server_validation_rejects_before_any_cuda_call():
    L = sinet.load()
    h = ctypes.c_void_p()
    ten = (sinet.TenantC * 1)()
    ten[0].table = 0x1000
    ten[0].params = sinet.HistParams(0, 1, 10).c()
    good = sinet.ServerConfigC(1 << 20, 16, 100)
    for cfg in (sinet.ServerConfigC(1 << 19, 16, 100), sinet.ServerConfigC(1 << 20, 0, 100),
                sinet.ServerConfigC(1 << 20, 5000, 100), sinet.ServerConfigC(1 << 20, 16, 0)):
        assert L.sinet_server_create(ctypes.byref(cfg), ten, 1, ctypes.byref(h)) == 1
    assert L.sinet_server_create(ctypes.byref(good), ten, 0, ctypes.byref(h)) == 1
    bad = (sinet.TenantC * 1)()
    bad[0].params = sinet.HistParams(0, 1, 10).c()  # no table
    assert L.sinet_server_create(ctypes.byref(good), bad, 1, ctypes.byref(h)) == 1
    bad[0].table = 0x1000
    bad[0].params = sinet.HistParams(0, 0, 10).c()  # zero bin width
    assert L.sinet_server_create(ctypes.byref(good), bad, 1, ctypes.byref(h)) == 1
    bad[0].params = sinet.HistParams(0, 1, 10, strategy="sort_reduce").c()  # not run by the server
    assert L.sinet_server_create(ctypes.byref(good), bad, 1, ctypes.byref(h)) == 8
    t = ctypes.c_uint64()
    assert L.sinet_server_submit(None, 0, None, None, None, None, 0, ctypes.byref(t)) == 1
    assert L.sinet_server_wait(None, 1, 0, None) == 1
    assert L.sinet_server_drain(None, 0) == 1
    assert L.sinet_server_destroy(None) == 0


def _toggle_lookup(img, lay, addrs):
    """The shared-memory toggle lookup of the kernels, replayed on the host."""
    desc = img[lay["off_desc"]: lay["off_desc"] + 4 * (1 << lay["desc_bits"])].view(np.uint32)
    blocks = img[lay["off_blocks"]: lay["off_desc"]].view(np.uint32).reshape(-1, 4)
    shift = 32 - lay["desc_bits"]
    a = addrs.astype(np.uint64)
    d = desc[(a >> np.uint64(shift)).astype(np.int64)].astype(np.uint64)
    off = a & np.uint64((1 << shift) - 1)
    form = lay["max_blocks"] >> 8
    if form == 0:  # consecutive blocks: first (bits 0-23), count (bits 24-27)
        first = (d & np.uint64(0xFFFFFF)).astype(np.int64)
        nb = ((d >> np.uint64(24)) & np.uint64(0xF)).astype(np.int64)
        idx = [np.where(nb > k, first + k, -1) for k in range(int(nb.max()))]
    else:  # one or two independent block indices (bits 0-14, 15-29)
        idx = [(d & np.uint64(0x7FFF)).astype(np.int64)]
        if form == 2:
            idx.append(((d >> np.uint64(15)) & np.uint64(0x7FFF)).astype(np.int64))
    for ix in idx:
        assert ix.max() < len(blocks)  # every block read stays in the staged region
    state = (d >> np.uint64(31)).astype(np.uint8)
    for ix in idx:
        use = ix >= 0
        b = blocks[np.where(use, ix, 0)].astype(np.uint64)  # toggle offsets minus one
        assert np.all(b < 2 ** 31)
        par = ((off[:, None] >= b + np.uint64(1)).sum(axis=1) & 1).astype(np.uint8)
        state ^= np.where(use, par, 0).astype(np.uint8)
    # the kernels' form: bit 31 of desc XOR every (stored - off) mod 2^32;
    # forms 1 and 2 skip block index 0 (all padding: its four equal
    # differences XOR to zero), so check that skipping it changes nothing
    assert np.all(blocks[0] == 0x7FFFFFFF)
    x = d.copy()
    x_skip = d.copy()
    for ix in idx:
        use = ix >= 0
        b = blocks[np.where(use, ix, 0)].astype(np.uint64)
        diff = (b - off[:, None] + np.uint64(1 << 32)) & np.uint64(0xFFFFFFFF)
        v = diff[:, 0] ^ diff[:, 1] ^ diff[:, 2] ^ diff[:, 3]
        x ^= np.where(use, v, np.uint64(0))
        x_skip ^= np.where(use & ((ix > 0) if form != 0 else use), v, np.uint64(0))
    assert np.array_equal(x, x_skip)
    assert np.array_equal(((x >> np.uint64(31)) & np.uint64(1)).astype(np.uint8), state)
    return state


@pytest.mark.parametrize("seed", range(6))
def test_toggle_form_equals_oracle(orc, seed):
    rng = random.Random(100 + seed)
    net, ln = _random_table(rng, rng.randint(0, 60))
    if seed == 0:
        net, ln = net[:0], ln[:0]
    addrs = _edge_addrs(net, ln, rng, extra=3000)
    img, lay = sinet.sinet_prefix_table_image(net, ln)
    assert lay["iv_bytes"] % 16 == 0 and lay["off_desc"] % 16 == 0 and lay["iv_bytes"] <= len(img)
    want = (orc.classify(net, ln, addrs, np.zeros_like(addrs)) & 1) if len(net) else np.zeros(len(addrs), np.uint8)
    assert np.array_equal(_toggle_lookup(img, lay, addrs), want)


@pytest.mark.parametrize("want_form", [0, 1, 2])
def test_toggle_forms_equal_oracle(orc, want_form):
    """Tables built to need one block per bucket, two, or a variable count."""
    rng = random.Random(7 + want_form)
    base = 0x0A000000
    if want_form == 1:
        net = [base + (i << 20) for i in range(8)]
        ln = [16] * 8
    elif want_form == 2:   # 5-8 toggles crowd one /14 bucket
        net = [base + (i << 12) for i in range(4)]
        ln = [24] * 4
    else:                  # twenty /32 hosts in one /14 bucket
        net = [base + 7 * i for i in range(20)]
        ln = [32] * 20
    net, ln = np.array(net, np.uint32), np.array(ln, np.uint8)
    img, lay = sinet.sinet_prefix_table_image(net, ln)
    assert lay["iv_fits_smem"] == 1 and lay["max_blocks"] >> 8 == want_form
    addrs = np.concatenate([_edge_addrs(net, ln, rng, 2000),
                            np.arange(base - 8, base + 400, dtype=np.uint32)])
    want = orc.classify(net, ln, addrs, np.zeros_like(addrs)) & 1
    assert np.array_equal(_toggle_lookup(img, lay, addrs), want)


def test_toggle_form_on_workload_tables(orc):
    rng = random.Random(9)
    for key in ("tiny", "day", "heavy"):
        w = gen.WORKLOADS[key]
        net, ln = gen.make_table(w.table, w.seed)
        img, lay = sinet.sinet_prefix_table_image(net, ln)
        assert lay["iv_fits_smem"] == 1 and (lay["max_blocks"] & 0xFF) <= 2
        r = gen.make_records(gen.scaled(w, 50_000).records, w.seed, net, ln)
        addrs = np.concatenate([r["src"], r["dst"], _edge_addrs(net[:200], ln[:200], rng, 2000)])
        want = orc.classify(net, ln, addrs, np.zeros_like(addrs)) & 1
        assert np.array_equal(_toggle_lookup(img, lay, addrs), want)


def test_too_dense_bucket_uses_global_intervals():
    """A bucket needing more than 15 toggle blocks at every bucket width: the
    shared-memory form is not offered (lookups use global-memory intervals)."""
    net = np.array([0x0A000000 + 7 * i for i in range(80)], np.uint32)
    ln = np.full(80, 32, np.uint8)
    img, lay = sinet.sinet_prefix_table_image(net, ln)
    assert lay["iv_fits_smem"] == 0


def test_toggle_lookup_property(orc):
    """Property test (hypothesis): any list of up to 60 prefixes, host bits
    set, lengths /0-/32 with duplicates and nesting; the compiled image's
    lookup replayed on the host equals the oracle's loop over every entry at
    every prefix edge, its neighbours and random addresses."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    entry = st.tuples(st.integers(0, 2 ** 32 - 1), st.integers(0, 32))

    @hyp.settings(max_examples=120, deadline=None, derandomize=True)
    @hyp.given(st.lists(entry, min_size=1, max_size=60), st.integers(0, 2 ** 31))
    def check(entries, seed):
        net = np.array([e[0] for e in entries], np.uint32)
        ln = np.array([e[1] for e in entries], np.uint8)
        addrs = _edge_addrs(net, ln, random.Random(seed), extra=64)
        img, lay = sinet.sinet_prefix_table_image(net, ln)
        want = (orc.classify(net, ln, addrs, np.zeros_like(addrs)) & 1).astype(np.uint8)
        if lay["iv_fits_smem"]:
            assert np.array_equal(_toggle_lookup(img, lay, addrs), want)
        t = sinet.sinet_compile_prefix_table(net, ln)
        got = _member_index(t["lo"], t["hi"], t["index"], t["index_bits"], addrs)
        assert np.array_equal(got, want.astype(bool))

    check()


def test_ctypes_layouts_and_constants_match_the_header(tmp_path):
    """The binding's ctypes mirrors and constants equal what a C compiler
    makes of include/sinet.h: every struct's size and field offsets, and
    every enum and flag value."""
    import ctypes
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    structs = {"sinet_hist_params": sinet.HistParamsC, "sinet_hist_out": sinet.HistOutC,
               "sinet_batch_slice": sinet.BatchSliceC, "sinet_tenant": sinet.TenantC,
               "sinet_server_config": sinet.ServerConfigC, "sinet_request_info": sinet.RequestInfoC,
               "sinet_server_counters": sinet.ServerCountersC}
    consts = {f"SINET_STRAT_{k.upper()}": v for k, v in sinet.STRATEGIES.items()}
    consts.update({f"SINET_LOOKUP_{k.upper()}": v for k, v in sinet.LOOKUPS.items()})
    consts.update({name: code for code, name in sinet.STATUS.items()})
    consts.update({"SINET_HINT_TIME_SORTED": sinet.HINT_TIME_SORTED, "SINET_HINT_TUNE": sinet.HINT_TUNE,
                   "SINET_BATCH_AUTOTUNE": sinet.BATCH_AUTOTUNE,
                   "SINET_DIR_OUT": sinet.DIR_OUT, "SINET_DIR_IN": sinet.DIR_IN})
    # every enum member and flag the header defines has a binding constant
    import re

    with open(os.path.join(ROOT, "include", "sinet.h")) as f:
        header = f.read()
    declared = set(re.findall(r"\b(SINET_(?:STRAT|LOOKUP|ERR)_[A-Z0-9_]+)\s*=", header)) | {"SINET_OK"}
    declared |= set(re.findall(r"#define (SINET_(?:HINT|DIR|BATCH)_[A-Z0-9_]+)", header))
    assert declared <= set(consts), sorted(declared - set(consts))
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sinet.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    for name in consts:
        lines.append(f'  printf("{name} %lld\\n", (long long){name});')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, f"{cname}.{fname}"
    for name, v in consts.items():
        assert int(got[name]) == v, name
