"""bench.py's reference arm on the host (no GPU): the command line the benchmark contract uses prints
one JSON line with the contract's keys, on the default workload and plan."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_prints_one_contract_line():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "1")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "amplitudes/s" and d["value"] > 0
    assert d["config"]["workload"] == "grid6x6_d14_s10_open6_sa"
    assert d["config"]["amplitudes_per_gpu"] == 64 and d["config"]["slices"] == 1024
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_sliced_workload_plans():
    d = _run("--impl", "reference", "--workload", "sliced", "--steps", "1", "--warmup", "1")
    assert d["config"]["workload"] == "grid4x5_d12_s6_amp256_checkpoint"
    d = _run("--impl", "reference", "--workload", "sliced", "--plan", "level-aware", "--steps", "1", "--warmup", "1")
    assert d["config"]["workload"] == "grid4x5_d12_s6_amp256_levelplan"
    d = _run("--impl", "reference", "--workload", "sliced", "--plan", "greedy", "--steps", "1", "--warmup", "1")
    assert d["config"]["workload"] == "grid4x5_d12_s6_amp256"
