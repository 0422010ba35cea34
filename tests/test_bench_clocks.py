"""The benchmark's clock record on CPU, with a stand-in nvidia-smi on PATH that
prints rows of the query for two GPUs: only this GPU's rows count (matched by
PCI bus id); the record holds the median SM clock, the maximum clock, the
throttle reasons seen active (thermal and hardware slowdowns included, so a
throttled run can be rejected) and the sample count; without nvidia-smi the
record says so."""
import os
import stat
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

ROWS = """0, 00000009:01:00.0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
1, 00000019:01:00.0, 1200, 2070, 310.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active
0, 00000009:01:00.0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, 00000009:01:00.0, 2040, 2070, 1401.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active
"""


def fake_smi(tmp_path, monkeypatch):
    (tmp_path / "rows.csv").write_text(ROWS)
    exe = tmp_path / "nvidia-smi"
    exe.write_text(f"#!/bin/sh\ncat {tmp_path / 'rows.csv'}\nexec sleep 30\n")
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")


def sample(bus):
    c = bench.ClockSampler(bus)
    c.start()
    return c.stop()


def test_rows_of_this_gpu(tmp_path, monkeypatch):
    fake_smi(tmp_path, monkeypatch)
    r = sample("0009:01:00.0")
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    r = sample("0019:01:00.0")
    assert r["reasons"] == ["hw_thermal_slowdown"] and r["sm_mhz"] == 1200.0 and r["samples"] == 1


def test_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    r = sample(None)
    assert r["samples"] == 0 and r["reasons"] == ["nvidia-smi unavailable"]
