"""Host-side rules of bench.py's JSON line that need no GPU: the DRAM traffic
of the roofline comes from the committed ncu record only while the kernel
sources are those it was captured at, and the record names the kernel the
roofline reports."""
import json
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_record_applies_only_at_its_sources():
    # the committed record names the kernel the headline roofline reports
    # (N = 4096) and the profile it comes from; its bytes are reported only
    # while the kernel sources hash to the one it was captured at
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    r = rec["k_persistent<12>"]
    assert r["dram_bytes_per_launch"] > 0
    assert os.path.exists(os.path.join(ROOT, r["source"]))
    current = r["kernel_sources_sha256_16"] == bench.kernel_sources_hash()
    assert bench.ncu_traffic("k_persistent<12>") == (r["dram_bytes_per_launch"] if current else None)
    assert bench.ncu_traffic("k_no_such_kernel") is None


def test_traffic_is_null_once_the_sources_change(tmp_path, monkeypatch):
    # a copy of the tree whose kernel sources differ by one byte: the record
    # no longer applies and the line carries null
    tree = tmp_path / "t"
    (tree / "paper_1711_08604_gb300" / "csrc").mkdir(parents=True)
    (tree / "profiles").mkdir()
    for f in ("afd_kernels.cu", "afd_device.cuh", "afd_fft.cuh", "afd_internal.h"):
        shutil.copy(os.path.join(ROOT, "paper_1711_08604_gb300", "csrc", f), tree / "paper_1711_08604_gb300" / "csrc" / f)
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.json"), tree / "profiles" / "traffic.json")
    monkeypatch.setattr(bench, "ROOT", str(tree))
    assert bench.ncu_traffic("k_persistent<12>") is not None
    with open(tree / "paper_1711_08604_gb300" / "csrc" / "afd_fft.cuh", "a") as fh:
        fh.write("\n")
    assert bench.ncu_traffic("k_persistent<12>") is None
    (tree / "profiles" / "traffic.json").write_text("not json")
    assert bench.ncu_traffic("k_persistent<12>") is None
