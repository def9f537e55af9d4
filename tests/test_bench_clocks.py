"""bench.py's clock record: nvidia-smi is started before the timed steps and
its first sample awaited (its start-up stays out of the timed region), and
the record holds only the samples taken from then on, at least one of them.
Runs against a stand-in nvidia-smi on PATH; no GPU."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!{python}
import sys, time
time.sleep(0.3)  # slow start-up, as on a fresh machine
# the first sample (taken before the timed region) carries a clock that must
# not reach the record
line = "0, {{sm}}, 2070, 500.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
print(line.format(sm=100), flush=True)
while True:
    time.sleep(0.2)
    print(line.format(sm=2070), flush=True)
"""


@pytest.fixture()
def bench_module():
    sys.path.insert(0, ROOT)
    import bench
    yield bench


def test_sampler_settles_before_the_timed_region(bench_module, tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.format(python=sys.executable))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    s = bench_module.ClockSampler(0)
    t0 = time.time()
    s.start()
    assert time.time() - t0 >= 0.3  # start() waited for the first sample
    assert s.mark == len(s.lines) >= 1
    time.sleep(0.05)  # a timed region shorter than the sampling interval
    rec = s.stop()
    assert rec["samples"] >= 1
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_sampler_without_nvidia_smi(bench_module, tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench_module.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
