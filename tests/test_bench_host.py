"""Host logic of bench.py that needs no GPU: the recorded DRAM traffic is
reported only for the kernel code it was captured on."""
from __future__ import annotations

import os
import shutil

import bench


def test_code_only_ignores_comments_and_layout():
    a = "int f(int x) {  // add one\n    return x + 1; /* done */\n}\n"
    b = "int f(int x) {\n  /* a longer\n     comment */ return x + 1;\n}"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(a.replace("x + 1", "x + 2"))


def test_recorded_traffic_follows_the_code_hash():
    # every record is reported exactly while its kernel's code hashes to the
    # record's key; records for other workloads or kernels are absent
    with open(os.path.join(bench.ROOT, "profiles", "traffic.txt")) as f:
        recs = [dict(kv.split("=", 1) for kv in line.split()) for line in f
                if line.strip() and not line.startswith("#")]
    assert recs
    for r in recs:
        want = float(r["bytes_per_launch"]) if r["source"] == bench.kernel_source_hash(r["kernel"]) else None
        assert bench.recorded_traffic(r["kernel"], r["workload"]) == want
        assert bench.recorded_traffic(r["kernel"], "no-such-workload") is None
    assert bench.recorded_traffic("k_batch", "day-400M-diurnal-sorted") is None


def test_code_change_drops_the_record(tmp_path, monkeypatch):
    # a copy of the sources with one code token changed hashes differently,
    # and the record keyed to the original code is no longer reported
    csrc = os.path.join(bench.ROOT, "paper_2106_12863_gb300", "csrc")
    root = tmp_path / "repo"
    dst = root / "paper_2106_12863_gb300" / "csrc"
    shutil.copytree(csrc, dst, ignore=shutil.ignore_patterns("*.o"))
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    before = bench.kernel_source_hash("k_fused_tile")
    (root / "profiles" / "traffic.txt").write_text(
        f"kernel=k_fused_tile workload=day source={before} bytes_per_launch=12\n"
        f"kernel=k_fused_owner workload=day source={bench.kernel_source_hash('k_fused_owner')} "
        "bytes_per_launch=10\n")
    assert bench.recorded_traffic("k_fused_tile", "day") == 12
    f = dst / "fused.cu"
    f.write_text(f.read_text() + "\n// a trailing comment changes nothing\n")
    assert bench.kernel_source_hash("k_fused_tile") == before
    f.write_text(f.read_text().replace("ta.margin", "ta.margin + 0", 1))
    assert bench.kernel_source_hash("k_fused_tile") != before
    assert bench.recorded_traffic("k_fused_tile", "day") is None
    # the owner kernel's sources do not include fused.cu: its record stands
    assert bench.recorded_traffic("k_fused_owner", "day") == 10
