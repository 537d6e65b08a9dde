"""bench.py's reference arm (the oracle on the host cores) keeps the one-line
JSON contract, and under a multi-rank launch only rank 0 prints it.  CPU
only: the reference arm never touches a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = _run(None, "--steps", "1", "--warmup", "0", "--ref-budget", "2", "--cpu-cores", "2")
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "Gpixel/s labeled (bit-exact)" and d["unit"] == "Gpixel/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["dtype"] == "u8" and d["data"] == "synthetic"
    assert "10980x10980" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    lines = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "1", "--warmup", "0",
                 "--gpus", "2")
    assert lines == []


def test_reference_arm_uint16_scene():
    """--dtype u16: the oracle pool shares the uint16 reflectance scene."""
    lines = _run(None, "--dtype", "u16", "--steps", "1", "--warmup", "0", "--ref-budget", "2",
                 "--cpu-cores", "2")
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["dtype"] == "u16" and d["value"] > 0
    assert "uint16" in d["config"]["workload"]
    assert d["cpu_baseline"]["cores"] == 2 and d["cpu_baseline"]["value"] == d["value"]
