"""bench.py's reference arm: the oracle timed on the host cores, on the small
sphere workload and on the default (stress) workload's bounded sample. It
prints one JSON line with the keys of the benchmark contract; under torchrun
only rank 0 works and prints, the others exit 0 without output."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, "bench.py", "--impl", "reference", "--workload", "spheres", "--steps", "2", "--warmup", "3"]


def _run(cmd=CMD, **env):
    return subprocess.run(cmd, cwd=ROOT, env=dict(os.environ, **env), capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_the_contract_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["unit"] == "Gfrag/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["ms_per_step"] > 0 and line["data"] == "synthetic"
    assert line["config"]["workload"] == "spheres8_256_d6"
    assert line["config"]["fragments_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_reference_arm_default_workload_is_the_stress_sample():
    """The default line's reference arm: the stress workload's configuration,
    each step one bounded triangle sample timed by the oracle."""
    r = _run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "Gfrag/s" and line["value"] > 0
    assert line["config"]["workload"] == "stress16M_axis3_d11_4k" and line["config"]["depth"] == 11
    assert "1024th triangle" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0
