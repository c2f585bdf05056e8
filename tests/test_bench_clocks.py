"""Host logic of bench.py's clock sampler (no GPU): a stand-in for the sampling
process writes timestamped lines; only the samples inside the marked timed regions
count, and the throttle reasons among them are reported."""
import datetime
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _line(t, mhz, hw_slowdown=False, power_cap=False):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    act = lambda b: "Active" if b else "Not Active"
    return (f"{ts}, {mhz}, 2070, 900.0, 0x0, {act(hw_slowdown)}, Not Active, Not Active, "
            f"{act(power_cap)}\n")


@pytest.fixture
def sampler(monkeypatch):
    import bench
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: _FakeProc())
    with monkeypatch.context() as m:           # skip only the start-up pause
        m.setattr(bench.time, "sleep", lambda s: None)
        return bench.ClockSampler(0)


def test_only_samples_inside_timed_regions_count(sampler):
    t0 = time.time()
    with sampler:
        time.sleep(0.05)
    time.sleep(0.2)                             # an untimed gap
    with sampler:
        time.sleep(0.05)
    (r0, r1), (r2, r3) = sampler.regions
    with open(sampler.path, "w") as f:
        f.write(_line(r0 - 1.0, 300, hw_slowdown=True))    # idle, before: ignored
        f.write(_line((r0 + r1) / 2, 2070))
        f.write(_line((r1 + r2) / 2, 345))                   # between regions: ignored
        f.write(_line((r2 + r3) / 2, 2055, power_cap=True))
        f.write("malformed line\n")
    s = sampler.summary()
    assert s["samples"] == 2 and s["regions"] == 2
    assert s["sm_mhz"] == pytest.approx((2070 + 2055) / 2)
    assert s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    assert r0 >= t0
    assert not os.path.exists(sampler.path)


def test_no_sample_in_a_region_is_reported(sampler):
    with sampler:
        pass
    with open(sampler.path, "w") as f:
        f.write(_line(time.time() + 10.0, 2070))
    assert sampler.summary()["reasons"] == ["no samples"]
