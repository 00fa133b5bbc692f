"""bench.py's command-line contract on a machine without a GPU (CPU only)."""
import json
import os
import subprocess
import sys

import pytest
import torch


def _run_bench(*args):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], capture_output=True,
                       text=True, timeout=600, cwd=root)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return r.returncode, [json.loads(l) for l in lines], r.stderr


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the oracle on the host cores and prints
    one JSON line with the main arm's metric, unit and config."""
    rc, out, err = _run_bench("--impl", "reference", "--steps", "1", "--warmup", "3", "--ref-stamps", "60")
    assert rc == 0, err[-2000:]
    assert len(out) == 1
    d = out[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "stamps/s"
    assert d["metric"].startswith("stamps fitted/sec") and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("uniform-48px") and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_gpu_arm_fails_loudly_without_a_gpu():
    """With no CUDA device the main arm exits non-zero and prints no number."""
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, out, _ = _run_bench("--steps", "1", "--warmup", "3", "--no-cpu")
    assert rc != 0 and out == []
