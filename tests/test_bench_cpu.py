"""Host logic of the benchmark (CPU): its defaults, and the committed ncu traffic figures,
which it reports only while they were taken on the current kernel sources."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_defaults_finish_quickly_and_keep_the_timing_rules(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "ours" and a.workload == "doppler2d"
    assert a.warmup >= 3 and a.steps >= 1
    assert bench.FLUSH_BYTES > 129e6          # L2 eviction buffer larger than the 129 MB L2


def test_committed_traffic_matches_the_kernel_sources():
    data = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    key = "staged_c64p_x32_f8v1w7t14e@doppler2d_256x256x32"
    assert data[key]["kernel_sha"] == bench.kernel_hash()
    e = bench.profiled_entry(*key.split("@"))
    assert e["dram_bytes_per_launch"] > 0 and e["l2_bytes_per_launch"] > e["dram_bytes_per_launch"]
    assert bench.profiled_traffic(*key.split("@")) == e["dram_bytes_per_launch"]


def test_stale_or_missing_traffic_is_not_reported(monkeypatch):
    key = ("staged_c64p_x32_f8v1w7t14e", "doppler2d_256x256x32")
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.profiled_entry(*key) == {} and bench.profiled_traffic(*key) is None
    monkeypatch.undo()
    assert bench.profiled_entry("no_such_variant", key[1]) == {}
