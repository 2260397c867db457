"""bench.py's reference arm (the FP64 oracle timed on the host cores) prints
one JSON line with the contract's keys; under a multi-rank launch only rank 0
prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
       "--ref-blocks", "1"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run(CMD, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    d = json.loads(lines[-1])
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "train-points/s" and d["higher_is_better"] is True
    assert d["metric"] == "LMA fit+predict train-points/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("C4:")  # the default workload: the largest single-GPU one
    assert "first 1 of 2000 blocks" in d["cpu_baseline"]["sample"]


def test_reference_arm_other_ranks_are_silent():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []
