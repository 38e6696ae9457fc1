"""Host logic of bench.py: the clock record that decides whether a timed run is
kept.  ``ClockSampler.summary`` reads nvidia-smi's CSV samples, keeps those
inside the timed region's wall-clock window, and reports the median SM clock,
the highest maximum clock and every throttle reason active in the window."""
import datetime
import os
import tempfile

import bench


def _line(t, sm, smax, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([ts, "0", str(sm), str(smax), "900.0", "0x0"] + flags) + "\n"


def _sampler(lines, window):
    s = bench.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as fh:
        fh.writelines(lines)
    s.proc = object()            # samples were taken (no nvidia-smi process is started here)
    s.mark(*window)
    return s


def test_window_median_and_reasons():
    t0 = 1_700_000_000.0
    lines = [_line(t0 - 1.0, 1200, 2070, ("hw_slowdown",))]             # before the timed region
    lines += [_line(t0 + 0.05 * k, 2070 - (k % 2) * 30, 2070) for k in range(10)]
    lines += [_line(t0 + 0.2, 2055, 2070, ("sw_power_cap",))]
    lines += ["garbage line\n", _line(t0 + 5.0, 900, 2070, ("hw_thermal_slowdown",))]   # after it
    out = _sampler(lines, (t0, t0 + 0.5)).summary()
    assert out["samples"] == 11
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]


def test_throttle_inside_the_window_is_reported():
    t0 = 1_700_000_000.0
    lines = [_line(t0 + 0.05 * k, 1500, 2070, ("hw_thermal_slowdown",) if k == 3 else ()) for k in range(6)]
    out = _sampler(lines, (t0, t0 + 0.3)).summary()
    assert out["reasons"] == ["hw_thermal_slowdown"] and out["sm_mhz"] == 1500


def test_no_samples_and_no_tool():
    t0 = 1_700_000_000.0
    assert _sampler([], (t0, t0 + 1.0)).summary()["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)    # never entered: nvidia-smi was not started
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]
