"""bench.py's clock record on CPU: nvidia-smi rows (timestamp first) are kept
only inside the host window that brackets the timed steps, throttle reasons
seen there are reported, and a window with no sample falls back to the
nearest one."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _row(t, sm, reasons=()):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = ["Active" if nm in reasons else "Not Active" for nm in bench.CLOCK_REASONS]
    return [ts, " 0", " %d" % sm, " 2070", " 900.5", " 0x0"] + [" " + f for f in flags]


def test_window_median_and_reasons():
    t0 = 1_700_000_000.0
    rows = [_row(t0 - 0.3, 1200, ("hw_slowdown",)),        # before the window: ignored
            _row(t0 + 0.05, 2070), _row(t0 + 0.15, 2055, ("sw_power_cap",)), _row(t0 + 0.25, 2070),
            _row(t0 + 0.6, 900, ("hw_thermal_slowdown",))]  # after: ignored
    ck = bench.summarise_clock_rows(rows, t0, t0 + 0.3)
    assert ck["samples"] == 3
    assert ck["sm_mhz"] == 2070
    assert ck["sm_max_mhz"] == 2070
    assert ck["reasons"] == ["sw_power_cap"]
    assert ck["window_s"] == 0.3


def test_empty_window_takes_nearest_sample():
    t0 = 1_700_000_100.0
    rows = [_row(t0 - 1.0, 1500), _row(t0 + 0.12, 2040), _row(t0 + 2.0, 1000)]
    ck = bench.summarise_clock_rows(rows, t0, t0 + 0.05)
    assert ck["samples"] == 1 and ck["sm_mhz"] == 2040 and ck["reasons"] == []


def test_malformed_rows_are_skipped():
    t0 = 1_700_000_200.0
    rows = [["garbage"], _row(t0 + 0.01, 2070), ["2026/13/45 99:99:99.000"] + ["x"] * 9]
    ck = bench.summarise_clock_rows(rows, t0, t0 + 0.1)
    assert ck["samples"] == 1 and ck["sm_mhz"] == 2070
    assert bench.summarise_clock_rows([], t0, t0 + 0.1)["sm_mhz"] is None
