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


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_reports_median_clock_and_active_reasons():
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.out.write("0, 2070, 2070, 850.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1980, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 2070, 2070, 900.2, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "garbage line\n")
    res = cs.stop()
    assert res == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}


def test_clock_sampler_without_nvidia_smi_returns_none():
    cs = bench.ClockSampler(0)
    cs.proc = None
    assert cs.stop() is None
    os.unlink(cs.out.name)
