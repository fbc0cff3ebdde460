"""The reference arm of bench.py on the CPU: one JSON line with the keys the
benchmark contract names, for each single-GPU workload (small grid, two
steps), and rank > 0 exits without output."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
        "cpu_baseline", "e2e"}


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       capture_output=True, text=True, timeout=600, env=e)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


@pytest.mark.parametrize("workload", ["wave1024", "nls1024", "heat1024-neumann"])
def test_reference_arm_prints_one_contract_line(workload):
    lines = _run(["--impl", "reference", "--workload", workload, "--M", "64", "--steps", "2",
                  "--warmup", "1"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d), KEYS - set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["config"]["M"] == 64


def test_reference_arm_other_ranks_print_nothing():
    lines = _run(["--impl", "reference", "--M", "64", "--steps", "1", "--warmup", "1"],
                 env={"RANK": "1", "WORLD_SIZE": "2"})
    assert lines == []
