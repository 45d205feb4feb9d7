"""Host logic of bench.py's clock record: only the nvidia-smi samples stamped
inside the timed region count, and throttle reasons are collected from them
(no GPU: the sampler's lines are given directly)."""
import datetime

import bench


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _line(ts, clk, hw_slow="Not Active", power_cap="Not Active"):
    return (f"{ts.strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]}, 0, {clk}, 2070, 900.00, 0x0000000000000000, "
            f"{hw_slow}, Not Active, Not Active, {power_cap}")


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.proc = _DoneProc()
    c.lines = list(lines)
    return c


def test_only_samples_inside_the_window_count():
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    lines = [_line(t0 - datetime.timedelta(milliseconds=300), 345, hw_slow="Active"),  # idle, before
             _line(t0 + datetime.timedelta(milliseconds=100), 2070),
             _line(t0 + datetime.timedelta(milliseconds=300), 2055, power_cap="Active"),
             _line(t0 + datetime.timedelta(milliseconds=500), 2070),
             _line(t0 + datetime.timedelta(milliseconds=900), 500)]  # after
    r = _sampler(lines).stop(t0, t0 + datetime.timedelta(milliseconds=600))
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0
    assert r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]  # the hw_slowdown sample lies outside the window


def test_no_window_keeps_every_sample_and_bad_lines_are_skipped():
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    lines = [_line(t0, 2070), "garbage", _line(t0, "[N/A]"), _line(t0 + datetime.timedelta(seconds=1), 1800)]
    r = _sampler(lines).stop()
    assert r["samples"] == 2
    assert r["sm_mhz"] == (2070.0 + 1800.0) / 2


def test_a_window_without_samples_reports_none():
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    r = _sampler([_line(t0, 2070)]).stop(t0 + datetime.timedelta(seconds=5), t0 + datetime.timedelta(seconds=6))
    assert r["samples"] == 0 and r["sm_mhz"] is None
