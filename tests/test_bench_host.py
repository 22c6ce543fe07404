"""Host logic of bench.py without a GPU: the DRAM traffic figure comes from
the committed ncu summary only while the kernel sources hash to the value it
records, interpolated between its in-window and out-of-window figures; the
roofline peak comes from MEASURED_PEAKS.json or a stated fallback."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _summary_values():
    vals = {}
    for line in open(bench.PROFILE_SUMMARY).read().splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    return vals


def test_traffic_follows_the_committed_summary_while_the_sources_match():
    vals = _summary_values()
    if vals.get("kernel_source_sha256_16") != bench.kernel_source_sha():
        pytest.skip("kernel sources changed since the summary was taken")
    win = float(vals["dram_bytes_per_voxel_dft_window"])
    out = float(vals["dram_bytes_per_voxel_outside_window"])
    assert bench.stress_traffic_per_voxel(0.0) == pytest.approx(out)
    assert bench.stress_traffic_per_voxel(1.0) == pytest.approx(win)
    assert bench.stress_traffic_per_voxel(0.25) == pytest.approx(0.25 * win + 0.75 * out)


def test_traffic_is_null_for_other_kernel_sources(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert bench.stress_traffic_per_voxel(0.3) is None


def test_traffic_is_null_without_a_summary(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.stress_traffic_per_voxel(0.3) is None


def test_peak_from_measured_file_or_fallback(monkeypatch, tmp_path):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6791.4}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak_hbm() == (6791.4, "measured")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "nowhere"))
    assert bench.measured_peak_hbm() == (6800.0, "fallback")


def test_whole_job_rate_counts_every_rank():
    # two ranks, 5 steps of 1e9 voxel-steps each, 1000 ms (max over ranks)
    assert bench.whole_job_rate(2, 5, 1e9, 1000.0) == pytest.approx(10.0)
