"""The bench's clock record, on the CPU against a fake nvidia-smi: only the
samples taken after the sampler has started (during the timed steps) are
kept, their median SM clock is reported, and an active throttle reason is
named.  No GPU and no real nvidia-smi are involved."""
import os
import stat
import sys
import time

FAKE = r'''#!PYTHON
import sys, time
idle = "0, 100, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
busy = "0, 2000, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active\n"
sys.stdout.write(idle * 5)
sys.stdout.flush()
time.sleep(0.2)
for _ in range(3):
    sys.stdout.write(busy)
    sys.stdout.flush()
    time.sleep(0.02)
time.sleep(30)
'''


def test_clock_sampler_keeps_the_timed_samples(tmp_path, monkeypatch):
    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text(FAKE.replace("PYTHON", sys.executable))
    fake.chmod(fake.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    assert s.skip == 5  # the five samples taken before the timed region
    time.sleep(0.6)
    clk = s.stop()
    assert clk["samples"] == 3
    assert clk["sm_mhz"] == 2000.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
