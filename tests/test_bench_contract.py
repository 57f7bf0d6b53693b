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


def _bench_module():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_committed_ncu_summaries_match_the_kernel_sources():
    """The figures the bench line reads from profiles/ (DRAM traffic per cell
    of the FP32 step, ALU-roof counts of the FP16, BF16 and learned steps) were
    taken from the kernel sources as committed: each summary records the
    hash of its sources and is dropped (null in the line) when they differ."""
    bench = _bench_module()
    assert bench.kernel_traffic_per_cell() is not None
    pull4 = ("lbm_device.cuh", "lbm_kernels.cuh", "lbm_packed.cuh")
    closure = ("lbm_device.cuh", "lbm_closure.cu")
    for name, src in (("alu_k_pull4_d3q27_cumulant_f16.md", pull4),
                      ("alu_k_pull4_d3q27_cumulant_bf16.md", pull4),
                      ("alu_k_closure_pull_d3q27_128.md", closure)):
        for key in ("fp32_flop_per_cell", "fp32_lane_ops_per_cell", "thread_inst_per_cell"):
            assert bench.profile_value(name, key, src) is not None, (name, key)


def test_alu_roof_and_summary_arithmetic():
    bench = _bench_module()
    src = ("lbm_device.cuh", "lbm_closure.cu")
    roof = bench.alu_roof("alu_k_closure_pull_d3q27_128.md", 10000.0, 80.0, src)
    fpc = roof["flop_per_cell"]
    assert abs(roof["achieved"] - fpc * 1e4 * 1e6 / 1e12) < 1e-9
    assert abs(roof["frac"] - roof["achieved"] / 80.0) < 1e-12
    # lane-ops and instructions against the lane / issue rate, half the flop peak
    assert abs(roof["pipe_frac"] - roof["lane_ops_per_cell"] * 1e10 / 40e12) < 1e-12
    assert abs(roof["issue_frac"] - roof["inst_per_cell"] * 1e10 / 40e12) < 1e-12
    line = {"value": 31000.0, "roofline": {"frac": 1.05},
            "forms": {"f16_delta": {"mlups": 52000.0, "roofline_frac": 0.87,
                                    "u_rel_linf_vs_f64": 7e-4, "alu": roof},
                      "f16_delta_aa": {"mlups": 1.0, "roofline_frac": 0.8,
                                       "clocks": {"sm_mhz": 1845.0, "reasons": ["sw_power_cap"]}},
                      "f16_delta_et": {"mlups": 1.0, "roofline_frac": 0.99,
                                       "clocks": {"sm_mhz": 2032.0, "reasons": []}}},
            "batched": None, "learned": None, "cpu_baseline": None, "sustained": None}
    s = bench.summary(line, [30000.0, 31000.0, 32000.0])
    assert s["headline_window_median_mlups"] == 31000.0
    assert s["f16_delta_pull"]["alu_frac"] == round(roof["frac"], 3)
    assert s["f16_delta_inplace_frac"] == {"aa": 0.8, "et": 0.99}
    # the SM clock each in-place form ran at (sampled over its timing)
    assert s["f16_delta_inplace_sm_mhz"] == {"aa": 1845.0, "et": 2032.0}
    assert len(json.dumps(s)) < 1500
