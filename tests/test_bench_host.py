"""Host logic of bench.py on the CPU: the clock record's parsing and the rule
that sends a timed region back for one more measurement."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


class _FakeSmi:
    """Stands in for the nvidia-smi sampling process."""

    def __init__(self, lines):
        self.out = "\n".join(lines) + "\n"

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def _sample(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.5, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def _clocks(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeSmi(lines)
    return s.stop()


def test_clock_record_parsing():
    c = _clocks([_sample(2070, 2070), _sample(2055, 2070), _sample(1980, 2070, cap="Active"), "garbage"])
    assert c["samples"] == 3 and c["sm_mhz"] == 2055 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]
    assert not bench.clocks_rejected(c)


def test_rejection_rule():
    assert bench.clocks_rejected(_clocks([_sample(2070, 2070, hw="Active")]))
    assert bench.clocks_rejected(_clocks([_sample(1800, 2070, hwt="Active")]))
    assert bench.clocks_rejected(_clocks([_sample(2000, 2070, swt="Active")]))
    # far below the maximum with no reason: a leftover clock lock
    assert bench.clocks_rejected(_clocks([_sample(1200, 2070), _sample(1200, 2070)]))
    # below the maximum under the power cap: kept
    assert not bench.clocks_rejected(_clocks([_sample(1500, 2070, cap="Active")]))
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})
