"""The bench's host-side parts, on CPU: the reference arm's JSON line (the FP64 oracle timed on
the host cores) and the CPU baseline's sampling, both on a 4,096-particle sphere at 16^3 so
that they end in seconds.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--n", "4096", "--mesh", "16", "--steps", "2", "--warmup", "1"]


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return out.stdout


def test_reference_arm_json_line():
    lines = [ln for ln in run_bench(["--impl", "reference", *SMALL]).splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "evals/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["n_gpus"] == 1
    assert 1 <= d["steps"] <= 2 and d["steps_requested"] == 2
    assert d["ms_per_step"] == pytest.approx(1e3 / d["value"], rel=1e-9)
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert "N=4,096" in d["config"]["workload"] and "16^3" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["unit"] == d["unit"] and "4,096" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    # under torchrun only rank 0 times the oracle and prints; the others exit 0 without work
    assert run_bench(["--impl", "reference", *SMALL],
                     {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}).strip() == ""


def test_cpu_baseline_counts_the_cell_list_once():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2103_02046_gb300 import bunches as B

    x = B.uniform_sphere(4096, 1e-3 * (4096 / 16777216) ** (1 / 3), 3)
    cb = bench.cpu_baseline(x, 16, 2.0, {}, budget_s=2.0)
    assert cb["kind"] == "oracle" and cb["unit"] == "evals/s" and cb["value"] > 0
    assert cb["seconds_per_eval"] == pytest.approx(1.0 / cb["value"], rel=1e-12)
    assert cb["cores"] >= 1 and "cell list over all N once" in cb["sample"]
    assert np.isfinite(cb["seconds_per_eval"])
