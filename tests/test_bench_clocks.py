"""The bench's clock sampler: a fake nvidia-smi on PATH stands in for the
real one (no GPU here). Entering the sampler waits for its first sample;
the summary takes the median SM clock, the largest maximum clock and every
throttle reason seen, within an optional time window."""
import os
import stat
import sys
import time

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _fake_smi(tmp_path, lines, delay_s=0.0, period_s=0.05):
    body = "\n".join("echo '%s'; sleep %g" % (l, period_s) for l in lines)
    script = tmp_path / "nvidia-smi"
    script.write_text("#!/bin/sh\nsleep %g\n%s\nwhile true; do sleep 1; done\n" % (delay_s, body))
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_sampler_waits_for_its_first_sample_and_summarises(tmp_path, monkeypatch):
    rows = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows, delay_s=0.3) + os.pathsep + os.environ["PATH"])
    t0 = time.monotonic()
    with bench.ClockSampler(0) as clk:
        # the first sample came after the fake's 0.3 s start-up, before entering returned
        assert len(clk.lines) >= 1 and time.monotonic() - t0 >= 0.25
        time.sleep(0.5)
    s = clk.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_summary_keeps_only_the_window():
    clk = bench.ClockSampler(0)
    clk.lines = [(1.0, "0, 1500, 2070, 500, 0x0, Active, Not Active, Not Active, Not Active\n"),
                 (2.0, "0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active\n"),
                 (3.0, "0, 2040, 2070, 950, 0x0, Not Active, Not Active, Not Active, Not Active\n"),
                 (4.0, "garbled\n")]
    s = clk.summary(1.5, 3.5)
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 2}
    assert clk.summary()["reasons"] == ["hw_slowdown"]
    assert bench.ClockSampler(0).summary()["samples"] == 0


def test_sampler_without_nvidia_smi_reports_no_samples(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    with bench.ClockSampler(0, first_wait_s=0.2) as clk:
        pass
    assert clk.summary()["samples"] == 0
