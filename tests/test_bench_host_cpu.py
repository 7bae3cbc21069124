"""The benchmark's host-side bookkeeping on the CPU: the recorded DRAM
traffic is used only while the kernel sources it was taken on are unchanged
(comments aside), the clock samples reduce to the median SM clock and the
throttle reasons seen, and the roofline denominator comes from the measured
peaks file when there is one."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    """A copy of the 128^3 kernel sources under a temporary root."""
    for p in bench.KERNEL_SOURCES[128]:
        dst = tmp_path / p
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, p), dst)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _write_record(root, sha, per_grid=1000.0):
    (root / "profiles" / "fft3d_128cubed_dram_traffic.txt").write_text(
        "# DRAM traffic of one launch\n"
        f"kernel_source_sha256_16: {sha}\n"
        f"dram_bytes_per_grid: {per_grid}\n")


def test_traffic_used_only_on_the_same_source(fake_root):
    sha = bench.kernel_source_hash(128)
    _write_record(fake_root, sha, per_grid=1234.0)
    assert bench.recorded_traffic(128, 32) == pytest.approx(1234.0 * 32)
    # a comment or a blank line keeps the record
    src = fake_root / bench.KERNEL_SOURCES[128][0]
    src.write_text(src.read_text() + "\n// a note\n\n")
    assert bench.kernel_source_hash(128) == sha
    assert bench.recorded_traffic(128, 32) == pytest.approx(1234.0 * 32)
    # a change of code drops it
    src.write_text(src.read_text() + "static int unused_marker = 1;\n")
    assert bench.kernel_source_hash(128) != sha
    assert bench.recorded_traffic(128, 32) is None


def test_traffic_missing_or_malformed_record(fake_root):
    assert bench.recorded_traffic(128, 32) is None
    (fake_root / "profiles" / "fft3d_128cubed_dram_traffic.txt").write_text(
        f"kernel_source_sha256_16: {bench.kernel_source_hash(128)}\n")
    assert bench.recorded_traffic(128, 32) is None


class _FakeProc:
    stdout = iter(())

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_reduce_to_median_and_reasons():
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = [
        "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
        "1965, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
        "2055, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 10.0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "garbage",
    ]
    c = s.stop()
    assert c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3
    s.lines = ["1500, 2070, 700, Active, Not Active, Active, Not Active"]
    assert s.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop() is None
    s.proc = _FakeProc()
    assert s.stop() is None  # no samples


def test_measured_peaks_file_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6778.5}))
    assert bench.measured_peaks() == (6778.5, "measured")


def test_whole_job_rate_counts_every_rank():
    # 2 ranks x 32 grids x 10 steps in 20 ms: 32000 transforms/s
    assert bench.whole_job_rate(2, 32, 10, 20.0) == pytest.approx(32000.0)
