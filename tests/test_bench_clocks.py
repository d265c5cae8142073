"""The bench's clock record keeps only nvidia-smi samples taken inside the timed region
(by their own timestamps), so throttle reasons seen before or after it do not count."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


class _Thread:
    def join(self, timeout=None):
        pass


def _line(t, mhz, reasons):
    stamp = t.strftime("%Y/%m/%d %H:%M:%S.") + f"{t.microsecond // 1000:03d}"
    flags = ", ".join("Active" if r else "Not Active" for r in reasons)
    return f"{stamp}, 0, {mhz}, 2070, 900.0, 0x0, {flags}"


def test_samples_outside_the_timed_region_are_dropped():
    import bench
    c = bench.ClockSampler(0)
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    ms = lambda k: t0 + datetime.timedelta(milliseconds=k)
    c.lines = [_line(ms(-500), 1100, (1, 0, 0, 0)),      # before: a slowdown that must not count
               _line(ms(20), 2070, (0, 0, 0, 1)),        # inside, power cap
               _line(ms(40), 2055, (0, 0, 0, 0)),        # inside
               _line(ms(60), 2070, (0, 0, 0, 0)),        # inside
               _line(ms(900), 800, (0, 1, 0, 0)),        # after
               "garbage line"]
    c.window = (t0, ms(100))
    c.proc, c.thread = _Proc(), _Thread()
    out = c.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_no_nvidia_smi_reports_it():
    import bench
    c = bench.ClockSampler(0)
    c.proc = None
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
