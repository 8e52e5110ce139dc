"""The bench's clock record on the host: `bench.Clocks` samples `nvidia-smi` during the timed region
and reports the median SM clock, the maximum clock and every throttle reason seen active.  A stand-in
`nvidia-smi` on PATH prints known samples (one malformed, one unreadable) and then waits to be
terminated, as the real one does with `-lms`."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

FAKE = """#!/bin/sh
echo "0, 1965, 2070, 900.1, 0x4, Not Active, Not Active, Not Active, Active"
echo "0, 1980, 2070, 910.0, 0x0, Not Active, Not Active, Not Active, Not Active"
echo "garbage line"
echo "0, [N/A], 2070, 905.0, 0x0, Not Active, Not Active, Not Active, Not Active"
echo "0, 1950, 2070, 905.0, 0x0, Not Active, Active, Not Active, Not Active"
exec sleep 30
"""


def test_clock_samples_median_max_and_reasons(tmp_path, monkeypatch):
    import bench
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    c = bench.Clocks(0)
    c.start()
    assert c.proc is not None
    deadline = time.time() + 10
    while time.time() < deadline and open(c.path).read().count("\n") < 5:
        time.sleep(0.05)
    rec = c.stop()
    assert rec == {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0, "reasons": ["hw_thermal_slowdown", "sw_power_cap"],
                   "samples": 3}
    assert c.proc.poll() is not None        # the sampler was stopped


def test_no_sampler_gives_no_record(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))   # no nvidia-smi anywhere
    c = bench.Clocks(0)
    c.start()
    assert c.stop() is None
    assert not os.path.exists(c.path)       # its sample file is removed as well
