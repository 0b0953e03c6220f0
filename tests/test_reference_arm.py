"""The benchmark's reference arm on the CPU: ``bench.py --impl reference``
times the FP64 oracle on the host cores and prints one JSON line with the
same metric, unit and workload as the GPU arm, a ``cpu_baseline`` that
describes the run and an ``e2e`` with no transfers; under a multi-rank launch
only rank 0 runs and prints, the other ranks exit 0 without work."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env, *args):
    env = dict(os.environ, **extra_env)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        if k not in extra_env:
            env.pop(k, None)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    pytest.importorskip("torch")
    import bench
    r = _run({}, "--steps", "1", "--warmup", "3", "--workload", "water24k")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 3)
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == "water24k" and d["config"]["n_atoms"] == 24000
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    pytest.importorskip("torch")
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--gpus", "2", "--steps", "1",
             "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_default_workload_is_the_3m_box():
    """With no flags the bench (and its reference arm) times the largest
    single-GPU machine, the 3,000,000-atom Ewald workload."""
    import bench
    args = bench.make_parser().parse_args([])
    assert args.workload == "water3m" and args.gpus == 1 and args.sub_blocks
    desc, fn = bench.workloads()["water3m"]
    assert "3,000,000" in desc
