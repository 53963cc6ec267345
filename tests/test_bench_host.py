"""Host-side logic of bench.py that needs no GPU: the clock record taken
during the timed region (median SM clock, max clock, active throttle reasons)
from the CSV that nvidia-smi writes."""
import os
import tempfile

import bench


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _stop_with(lines):
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = _DoneProc(), path
    out = s.stop()
    assert not os.path.exists(path)  # the sampler removes its file
    return out


def test_clock_record_median_max_and_reasons():
    na, a = "Not Active", "Active"
    rows = [f"0, {mhz}, 2070, 900.0, 0x0, {na}, {na}, {na}, {cap}"
            for mhz, cap in [(2070, na), (1980, a), (2070, na), (2055, na), (2070, na)]]
    out = _stop_with(rows + ["garbage line", ""])
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 5


def test_clock_record_reports_thermal_slowdown():
    na, a = "Not Active", "Active"
    rows = [f"0, 1500, 2070, 1400.0, 0x0, {a}, {na}, {a}, {na}"] * 3
    out = _stop_with(rows)
    assert out["sm_mhz"] == 1500.0
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    s = bench.ClockSampler(0)
    out = s.stop()  # never started: no nvidia-smi process
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
