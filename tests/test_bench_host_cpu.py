"""Host-side helpers of bench.py (no GPU): the clock record taken during
the timed region, the roofline peak, and the lookup of committed DRAM
traffic, which must only match summaries taken on the current kernels."""
import json
import os

import pytest

import bench


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(tmp_path, rows):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(", ".join(r) + "\n" for r in rows))
    s = bench.ClockSampler(0)
    s.proc, s.path = _DoneProc(), str(path)
    return s


def _row(sm, mx=2070, active="0x0", hw="Not Active", hwt="Not Active", swt="Not Active",
         pcap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", active, hw, hwt, swt, pcap]


def test_clocks_median_under_load_and_reasons(tmp_path):
    rows = [_row(345), _row(2070), _row(2070), _row(2055, pcap="Active"), _row(2070), _row(390)]
    c = _sampler(tmp_path, rows).stop()
    assert c["samples"] == 6
    assert c["sm_max_mhz"] == 2070
    assert c["sm_mhz"] == 2070          # idle samples (below half the top clock) left out
    assert c["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(str(tmp_path / "clocks.csv"))


def test_clocks_thermal_reasons_are_reported(tmp_path):
    rows = [_row(1800, hwt="Active"), _row(1790, swt="Active"), _row(1810, hw="Active")]
    c = _sampler(tmp_path, rows).stop()
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1800


def test_clocks_without_samples(tmp_path):
    assert _sampler(tmp_path, []).stop() is None
    s = bench.ClockSampler(0)
    assert s.stop() is None           # never started


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6783.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6783.5, "measured")
    (tmp_path / "MEASURED_PEAKS.json").unlink()
    assert bench.measured_peaks() == (6800.0, "fallback")


def _tree(tmp_path, kernel_text, name="batch_fwd.cu"):
    csrc = tmp_path / "paper_2505_21728_gb300" / "csrc"
    csrc.mkdir(parents=True, exist_ok=True)
    for f in bench.BATCH_SOURCES:
        if not (csrc / f).exists():
            (csrc / f).write_text("// " + f)
    (csrc / name).write_text(kernel_text)
    (tmp_path / "profiles").mkdir(exist_ok=True)


def test_traffic_only_for_the_current_kernel_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, "kernel v1")
    sha1 = bench.kernel_source_sha()
    (tmp_path / "profiles" / "k.md").write_text(
        "# summary\n"
        "bench-traffic: kernel=fwd workload=w8 sha=%s variant=0,0 bytes_per_launch=1572022272\n"
        "bench-traffic: kernel=inv workload=w8 sha=%s variant=2,0 bytes_per_launch=1.6e9\n"
        % (sha1, sha1))
    assert bench.ncu_traffic("fwd", "w8") == 1572022272
    assert bench.ncu_traffic("fwd", "w8", (12, 0, 0, 0.5)) == 1572022272
    assert bench.ncu_traffic("fwd", "w8", (4, 2, 0, 0.5)) == 1572022272     # same kernel
    assert bench.ncu_traffic("fwd", "w8", (12, 0, 2, 0.5)) is None   # another staging variant
    assert bench.ncu_traffic("inv", "w8", (4, 0, 2)) == 1600000000
    assert bench.ncu_traffic("fwd", "w8", (12, 0, 0, 0, 0.5)) == 1572022272  # layout 0
    assert bench.ncu_traffic("fwd", "w8", (12, 0, 0, 1, 0.5)) is None        # layout 1
    assert bench.ncu_traffic("fwd", "other") is None
    _tree(tmp_path, "kernel v1", name="secondary.cu")  # another kernel's source: no effect
    assert bench.kernel_source_sha() == sha1
    _tree(tmp_path, "kernel v2")      # the batch kernels changed since the capture
    assert bench.kernel_source_sha() != sha1
    assert bench.ncu_traffic("fwd", "w8") is None
