"""bench.py's clock sampler on CPU, against a stand-in for nvidia-smi that
prints the sampler's CSV fields: the median SM clock, the maximum, and the
throttle reasons seen in the timed region's samples."""
import os
import stat

import bench


def _fake_smi(tmp_path, lines, period=0.05):
    script = tmp_path / "nvidia-smi"
    body = [f"print({ln!r}, flush=True); time.sleep({period})" for ln in lines]
    script.write_text("\n".join(["#!/usr/bin/env python3", "import time", *body, "time.sleep(60)", ""]))
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def _row(sm, mx, hw="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.0, 0x0, {hw}, Not Active, Not Active, {cap}"


def test_sampler_reports_median_max_and_reasons(tmp_path, monkeypatch):
    d = _fake_smi(tmp_path, [_row(1000, 2070), _row(2070, 2070), _row(2060, 2070, cap="Active"),
                             _row(2070, 2070)])
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler("0").start()
    import time
    time.sleep(0.5)
    c = s.stop()
    # the first sample arrives before the timed region starts and is left out
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_sampler_keeps_the_last_sample_of_a_short_region(tmp_path, monkeypatch):
    d = _fake_smi(tmp_path, [_row(2070, 2070, hw="Active")], period=0.0)
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler("0").start().stop()
    assert c["samples"] == 1 and c["sm_mhz"] == 2070.0 and c["reasons"] == ["hw_slowdown"]


def test_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    assert bench.ClockSampler("0").start().stop() is None
