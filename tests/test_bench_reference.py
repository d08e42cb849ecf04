"""The reference arm of bench.py (the FP64 oracle on the host cores) runs on CPU: one JSON line
with the keys of the benchmark line, its e2e and cpu_baseline describing the same run; ranks
other than 0 do no work."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_line():
    r = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    assert j["unit"] == "Gcoef/s" and j["higher_is_better"] is True and j["value"] > 0
    assert (j["n_gpus"], j["steps"], j["warmup"]) == (1, 2, 1)
    assert abs(j["ms_per_step"] - j["config"]["coefs"] / j["value"] / 1e6) <= 1e-6 * j["ms_per_step"]
    assert j["vs_baseline"] is None and j["data"] == "synthetic" and j["dtype"] == "f64"
    assert j["config"]["workload"].startswith("mixed4-64-")
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == j["value"]
    e2e = j["e2e"]
    assert e2e == {"value": j["value"], "unit": j["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
