"""The bench.py output contract, checked on a host without a GPU: the
reference arm (the FP64 oracle on the host cores) prints one JSON line with
every key of the contract and the cuda arm's workload, and the cuda arm
fails loudly instead of falling back to the CPU when there is no device."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=timeout, cwd=ROOT)


def test_reference_arm_line():
    r = run_bench("--impl", "reference", "--steps", "2", "--warmup", "0", "--ref-edge", "8")
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["unit"] == "MLUPS" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["n_gpus"] == 1
    assert line["config"]["cells"] == 512 ** 3  # the cuda arm's workload, sampled
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "8^3" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_cuda_arm_fails_loudly_without_a_device():
    r = run_bench("--steps", "1", "--no-forms", "--no-e2e", "--no-cpu", "--no-batched",
                  "--no-learned", timeout=120)
    assert r.returncode != 0
    assert not r.stdout.strip().startswith("{")
