"""bench.py's reference arm (the oracle timed on the host cores) keeps the
one-JSON-line contract, on CPU: a small sample of the large workload, rank 0
prints, any other rank exits 0 without work."""
from __future__ import annotations

import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args, wall=None):
    env = {**os.environ, **(extra_env or {})}
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--scale", "8", "--steps", "2",
                        "--warmup", "3", *args], cwd=ROOT, capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    if wall is not None:
        wall.append(time.perf_counter() - t0)
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    wall = []
    lines = _run(None, wall=wall)
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("memory events/s characterized")
    assert d["unit"] == "events/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 3)
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert "large invocation" in d["config"]["workload"]
    # every claimed step ran, on the sample the workload names
    assert "reference sample per step" in d["config"]["workload"]
    assert d["steps"] * d["ms_per_step"] / 1e3 < wall[0]
    b = d["cpu_baseline"]
    assert b["kind"] == "oracle" and b["cores"] >= 1 and b["sample"] and b["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_names_the_workload_options():
    d = json.loads(_run(None, "--byte-addresses", "--history-scope", "1")[0])
    assert "byte-granular" in d["config"]["workload"] and "(site, work-item)" in d["config"]["workload"]


def test_reference_arm_other_ranks_exit_quietly():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_inputs_note_against_l2():
    sys.path.insert(0, ROOT)
    import bench
    full = 16 * (1 << 28) + 8 * (1 << 26) + 2 * (1 << 30) + 20 * (1 << 20)
    assert bench.inputs_note(full) == "device-resident, 7.00 GB > L2 (no flush)"
    assert "<= L2" in bench.inputs_note(64 << 20)


def test_all_cores_baseline_runs_oracle_replicas():
    """The all-cores CPU baseline: the oracle as it stands, one spawned process
    per core on its own sample, timed from the first start to the last finish."""
    sys.path.insert(0, ROOT)
    import bench
    b = bench.cpu_baseline_all_cores(10, {}, procs=2)
    assert b["kind"] == "oracle replicas" and b["cores"] == 2 and b["unit"] == "events/s"
    assert b["value"] > 0 and "2 processes" in b["sample"] and "65536 memory events" in b["sample"]


def test_reference_arm_refuses_other_workloads():
    d = json.loads(_run(None, "--workload", "serving")[0])
    assert d["impl"] == "reference" and "large invocation only" in d["unavailable"]
