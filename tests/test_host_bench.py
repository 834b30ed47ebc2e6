"""bench.py on the CPU: the reference arm (the CPU oracle on a bounded sample) — the
JSON line of the contract, the sample's codeword count against its closed form, the
other ranks of a multi-rank launch exiting without work — and the clock record taken
from nvidia-smi during the timed region."""

import json
import math
import os
import subprocess
import sys

from conftest import ROOT


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_line():
    lines = _run(None, "--steps", "2", "--warmup", "1", "--ref-levels", "5")
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "gpu_launches"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["unit"] == "codewords/s" and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["gpu_launches"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # [192,64] with three full-rank sets: every unit (g, j), g <= 5, enumerates C(64, g) combinations
    per_step = 3 * sum(math.comb(64, g) for g in range(1, 6))
    assert f"({per_step} codewords per step)" in d["config"]["sample"]
    assert d["config"]["n"] == 192 and d["config"]["k"] == 64


def test_reference_arm_other_ranks_exit_quietly():
    lines = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--gpus", "2", "--steps", "1", "--warmup", "1",
                 "--ref-levels", "3")
    assert lines == []


def test_clock_sampler_parses_nvidia_smi(tmp_path, monkeypatch):
    """The clock record of the bench line from nvidia-smi's CSV (a stand-in script on
    PATH prints it): median SM clock under load, the maximum, the throttle reasons that
    were active in any sample."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!/bin/sh\n"
        "echo '0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
        "echo '0, 1950, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
        "echo '0, 1965, 2070, 1385.2, 0x4, Not Active, Not Active, Not Active, Active'\n"
        "echo 'garbage line'\n"
        "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    import time

    import bench

    s = bench.ClockSampler(None)
    s.start()
    deadline = time.time() + 10
    while len(s.rows) < 3 and time.time() < deadline:
        time.sleep(0.05)
    rec = s.stop()
    assert rec == {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    import bench

    s = bench.ClockSampler(None)
    s.start()
    assert s.stop() is None


def test_reference_arm_loads_nothing_of_the_package():
    """The oracle arm computes with the oracle only: after a whole run the process has
    not mapped the package's library."""
    code = ("import runpy, sys\n"
            "sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', '--warmup', '0', '--ref-levels', '3']\n"
            "try:\n"
            "    runpy.run_path('bench.py', run_name='__main__')\n"
            "except SystemExit as e:\n"
            "    assert not e.code, e.code\n"
            "maps = open('/proc/self/maps').read()\n"
            "print('MAPPED' if 'libmdist' in maps else 'CLEAN')\n"
            "print('ORACLE' if 'liboracle' in maps else 'NO-ORACLE')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = r.stdout.split()
    assert "CLEAN" in out and "ORACLE" in out, r.stdout[-500:]
