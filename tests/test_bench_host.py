"""Host logic of bench.py that needs no GPU: the clock sampler, driven by a stand-in
`nvidia-smi` on PATH that prints rows in the query's CSV format."""
import importlib.util
import os
import stat
import sys
import time
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    sys.modules["bench_under_test"] = mod
    spec.loader.exec_module(mod)
    return mod


IDLE = "0, 1200, 2070, 150.00, 0x0, Not Active, Not Active, Not Active, Not Active"
BUSY = "0, 2070, 2070, 900.00, 0x4, Not Active, Not Active, Not Active, Active"


def _fake_smi(tmp_path, first, then):
    script = tmp_path / "nvidia-smi"
    script.write_text(
        "#!/bin/bash\n"
        f"echo '{first}'\n"
        "sleep 0.3\n"
        f"while true; do echo '{then}'; sleep 0.02; done\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_summarise_reasons_and_median():
    b = _bench()
    rows = [IDLE, BUSY, BUSY, "0, 1980, 2070, 1400.00, 0x8, Active, Not Active, Not Active, Not Active", "bad"]
    out = b.ClockSampler.summarise(rows)
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_sampler_keeps_only_the_timed_region(tmp_path, monkeypatch):
    b = _bench()
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, IDLE, BUSY) + os.pathsep + os.environ["PATH"])
    cs = b.ClockSampler(0)
    cs.start()
    assert cs.lines, "start() returns after the first sample"
    time.sleep(0.4)            # past the idle row
    t0 = time.perf_counter()
    time.sleep(0.2)
    t1 = time.perf_counter()
    out = cs.stop(t0, t1)
    assert out["samples"] >= 2
    assert out["sm_mhz"] == 2070.0 and out["reasons"] == ["sw_power_cap"]


def test_sampler_region_shorter_than_interval(tmp_path, monkeypatch):
    b = _bench()
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, IDLE, BUSY) + os.pathsep + os.environ["PATH"])
    cs = b.ClockSampler(0)
    cs.start()
    time.sleep(0.4)
    t0 = time.perf_counter()
    out = cs.stop(t0, t0)      # empty window: the first sample after t0 stands in
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0


def test_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    b = _bench()
    monkeypatch.setenv("PATH", str(tmp_path))
    cs = b.ClockSampler(0)
    cs.start()
    out = cs.stop(0.0, 1.0)
    assert out["reasons"] == ["nvidia-smi unavailable"]
