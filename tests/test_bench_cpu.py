"""The benchmark's reference arm (the oracle on the host cores) on CPU: one
JSON line with the contract's keys on rank 0, nothing on other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_prints_the_contract_line():
    lines = run_reference({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["config"]["workload"] == "c2_hea20_c64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    assert run_reference({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_oracle_timing_in_a_fresh_process():
    """The oracle baseline is timed in a child process, on all cores and on
    one (OpenMP held to one thread), in full steps of the headline workload."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    one = bench.oracle_timing(1.0, threads=1)
    assert one["cores"] == 1 and one["steps"] >= 1 and one["seconds"] > 0, one
    v = bench.oracle_line_values(W.config_c2(), one["steps"], one["seconds"])
    assert v["value"] > v["gate_equivalent"] > 0 and v["ms_per_step"] > 0
