"""Eq. 1 / Eq. 2 accounting helpers against the numbers the paper prints."""
import json
import os

import numpy as np

from paper_2604_06257_gb300 import counts

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))


def test_eq1_points_and_rates():
    for e in GOLD["eq1_points"]:
        if "frames" in e:
            got = counts.points(e["voxels"], e["channels"], e["compounding"], e["frames"])
        else:
            got = counts.throughput(e["voxels"], e["channels"], e["compounding"], e["frame_rate"])
        assert abs(got / e["printed"] - 1) <= e["rel_tol"], (e["cite"], got)
    # exact product of the benchmark configuration
    assert counts.points(251 * 251, 128, 1, 32) == 258_052_096


def test_throughput_from_runtime():
    for e in GOLD["throughput"]:
        got = e["points"] / e["seconds"]
        assert abs(got / e["printed"] - 1) <= e["rel_tol"]


def test_voxel_counts():
    for e in GOLD["voxel_counts"]:
        assert int(np.prod(e["dims"])) == e["printed"], e["cite"]


def test_memory_table3():
    e = GOLD["memory_table3"]
    m = counts.memory_table(e["voxels"], e["channels"], e["samples"], e["frames"], e["out_frames"])
    for k, gb in e["printed_gb"].items():
        assert abs(m[k] / 1e9 - gb) <= e["gb_tol"][k], (k, m[k])
    assert m["element_coords"] / 1e9 < 0.01
    assert m["arrival_times"] / 1e9 < 0.01
    assert abs(m["grid_coords"] / 1e9 - 0.01) < 0.005


def test_eq2_scaling():
    """Memory is linear in voxels x frames plus channels x samples x frames."""
    a = counts.memory_table(1000, 64, 100, 10)
    b = counts.memory_table(2000, 64, 100, 10)
    c = counts.memory_table(1000, 64, 100, 20)
    assert b["output"] == 2 * a["output"] and c["output"] == 2 * a["output"]
    assert c["channel_data"] == 2 * a["channel_data"]


def test_compulsory_bytes_doppler_benchmark_shape():
    # 256 x 256 px, 128 ch, 1 tx, 2048 samples, 32 frames, y + PD written
    b = counts.compulsory_bytes(65536, 128, 1, 2048, 32, write_y=True, write_pd=True)
    iq = 128 * 2048 * 32 * 8
    assert b == iq + 65536 * 4 + 65536 * 16 + 128 * 16 + 65536 * 32 * 8 + 65536 * 4
