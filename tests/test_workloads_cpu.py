"""Host-side checks of the benchmark's synthetic workloads and of its reference arm
(no GPU): the reduced adaptive meshes are complete and 2:1 balanced with the documented
sizes, and `bench.py --impl reference` prints one JSON line with the keys a bench
line carries."""
import json
import os
import subprocess
import sys

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _volume(leaves, dim, max_level):
    return float(np.sum((1.0 / (1 << leaves[:, 3].astype(np.int64))) ** dim))


def test_reduced_two_drop_workload_is_balanced():
    leaves, level, cfg, _ = bench.twodrops_workload(3, 7)
    assert level == 7 and cfg["Cn"] == 0.02 and cfg["rho_ratio"] == 100.0
    assert len(leaves) == 101_368
    assert abs(_volume(leaves, 3, level) - 1.0) < 1e-12
    assert len(synth.balance_leaves(leaves, 3, level)) == len(leaves)


def test_reduced_layer_workload_is_balanced_by_construction():
    leaves, level, cfg, _ = bench.layer_workload(4, 8)
    assert level == 8 and abs(cfg["Cn"] - 0.01) < 1e-15 and cfg["rho_ratio"] == 3.0
    assert len(leaves) == 1_632_128
    assert abs(_volume(leaves, 3, level) - 1.0) < 1e-12
    assert len(synth.balance_leaves(leaves, 3, level)) == len(leaves)


def test_reference_arm_prints_one_bench_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
