"""The bench's clock summary (host logic): samples written before the timed region
are left out, the median SM clock and the throttle reasons come from the rest."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

NA = "Not Active"


def _line(sm, reasons=()):
    flags = [("Active" if nm in reasons else NA)
             for nm in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")]
    return ", ".join(["0", str(sm), "2070", "812.50", "0x0000000000000000", *flags]) + "\n"


def _clocks(tmp_path, monkeypatch, lines, skip):
    monkeypatch.setenv("LM_CLOCKS_DIR", str(tmp_path))
    import bench

    c = bench.Clocks(0)
    with open(c.path, "w") as f:
        f.writelines(lines)
    c.skip = skip
    return c.summary()


def test_samples_before_the_region_are_left_out(tmp_path, monkeypatch):
    lines = [_line(345, ("hw_slowdown",)), _line(2070), _line(2055, ("sw_power_cap",)), _line(2070)]
    s = _clocks(tmp_path, monkeypatch, lines, skip=1)
    assert s["samples"] == 3
    assert s["sm_mhz"] == pytest.approx(2070.0)
    assert s["sm_max_mhz"] == pytest.approx(2070.0)
    assert s["reasons"] == ["sw_power_cap"]


def test_thermal_reason_inside_the_region_is_reported(tmp_path, monkeypatch):
    lines = [_line(2070), _line(1900, ("hw_thermal_slowdown", "sw_thermal_slowdown"))]
    s = _clocks(tmp_path, monkeypatch, lines, skip=0)
    assert s["samples"] == 2
    assert s["sm_mhz"] == pytest.approx(1985.0)
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_no_sample_in_the_region(tmp_path, monkeypatch):
    s = _clocks(tmp_path, monkeypatch, [_line(2070), "garbled\n"], skip=1)
    assert s["sm_mhz"] is None and s["reasons"] == ["no samples"]
