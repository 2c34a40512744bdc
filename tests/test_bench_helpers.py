"""Host logic behind fields of bench.py's JSON line, on the CPU: the
profiled DRAM traffic lookup (keyed by the device sources of the kernel kind
that ran) and the parsing of the nvidia-smi clock samples."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _profile_hash(kind):
    import re
    m = re.search(r"kernel_source_sha\[%s\]:\s*([0-9a-f]+)" % kind, open(bench.PROFILE).read())
    return m.group(1) if m else None


def test_profiled_traffic_matches_the_committed_profile():
    for kind, tile in (("plain", 1), ("pipelined", 12)):
        v = bench.profiled_traffic(tile, kind)
        if _profile_hash(kind) != bench.kernel_source_hash(kind):
            assert v is None, kind  # counters taken on other sources are not reported
            continue
        # one cold step reads the 18.87 MB of populations plus at most a few
        # percent of halo and frame sectors
        assert v is not None and 18.8e6 < v < 20.0e6, (kind, v)
    assert bench.profiled_traffic(9, "tma") is None       # kind not profiled
    assert bench.profiled_traffic(12345, "plain") is None  # tile not captured


def test_profiled_traffic_is_null_once_the_sources_change(monkeypatch, tmp_path):
    # a summary recorded on the current sources of both kinds: each kind's
    # figure is reported until that kind's own sources change
    prof = tmp_path / "profile.md"
    prof.write_text("kernel_source_sha[plain]: %s\nkernel_source_sha[pipelined]: %s\n"
                    "dram_bytes_per_launch[1]: 1.9e7\ndram_bytes_per_launch[13]: 1.95e7\n"
                    % (bench.kernel_source_hash("plain"), bench.kernel_source_hash("pipelined")))
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profiled_traffic(1, "plain") == 1.9e7
    assert bench.profiled_traffic(13, "pipelined") == 1.95e7
    real = bench.kernel_source_hash
    monkeypatch.setattr(bench, "kernel_source_hash",
                        lambda kind: "0" * 16 if kind == "plain" else real(kind))
    assert bench.profiled_traffic(1, "plain") is None
    assert bench.profiled_traffic(13, "pipelined") == 1.95e7


class _FakeSmi:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def _sampler(monkeypatch, lines):
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: _FakeSmi("\n".join(lines) + "\n"))
    return bench.ClockSampler(0)


def test_clock_samples_are_summarised(monkeypatch):
    row = "0, {sm}, 2070, 900.5, {act}, Not Active, Not Active, Not Active, {cap}, {util}"
    lines = [row.format(sm=s, act="0x0", cap="Not Active", util=u) for s, u in ((2070, 97), (2070, 88), (2055, 91))]
    lines.append(row.format(sm=1980, act="0x4", cap="Active", util=99))
    lines.append(row.format(sm=345, act="0x0", cap="Not Active", util=0))   # idle: not under load
    lines.append("garbage line")
    clk = _sampler(monkeypatch, lines).stop()
    assert clk == {"sm_mhz": 2062.5, "sm_max_mhz": 2070.0, "samples": 5, "samples_under_load": 4,
                   "reasons": ["sw_power_cap"]}


def test_clock_median_falls_back_to_all_samples_without_utilisation(monkeypatch):
    lines = ["0, %d, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active" % s for s in (2070, 2000, 2055)]
    clk = _sampler(monkeypatch, lines).stop()
    assert clk["sm_mhz"] == 2055 and clk["samples_under_load"] == 0


def test_thermal_and_hardware_slowdowns_are_reported(monkeypatch):
    lines = ["0, 1500, 2070, 1000, 0x48, Active, Not Active, Active, Not Active"]
    clk = _sampler(monkeypatch, lines).stop()
    assert clk["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_no_samples_gives_no_clock_record(monkeypatch):
    assert _sampler(monkeypatch, []).stop() is None


def test_peak_is_the_measured_copy_bandwidth_when_recorded():
    peak, kind = bench.measured_peak_hbm()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak > 1000
    else:
        assert (peak, kind) == (6800.0, "fallback")
