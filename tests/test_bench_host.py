"""Host logic of bench.py that needs no GPU: the clock sampler, driven by a stand-in
`nvidia-smi` on PATH that prints rows in the query's CSV format, and the reference arm (the
oracle on the host cores) on a small workload."""
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


def _run_reference(env_extra=None):
    import json
    import subprocess
    env = dict(os.environ)
    env.update(env_extra or {})
    cmd = [sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--workload", "cfg2_small",
           "--steps", "1", "--warmup", "3"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line():
    """The reference arm (the oracle on the host cores) prints one JSON line with the
    contract's keys; its e2e moves no bytes between host and device."""
    out = _run_reference()
    assert len(out) == 1
    d = out[0]
    # one complete oracle ground state is timed whatever --steps asks for: steps and
    # ms_per_step describe what was measured, and fit the run's wall time
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["requested"] == {"steps": 1, "warmup": 3}
    assert d["ms_per_step"] * d["steps"] <= 1e3 * d["wall_s"]
    assert d["unit"] == "ground states/s" and d["higher_is_better"] is True and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    b = _bench()
    from ddinputs import WORKLOADS
    assert d["config"]["workload"] == b.workload_label(WORKLOADS["cfg2_small"])   # the GPU arm's label
    assert cb["inner_iters_total"] > 0 and cb["outer_iters"] > 0


def test_reference_arm_other_ranks_exit_quietly():
    assert _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
