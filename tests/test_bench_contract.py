"""bench.py on the CPU: the reference arm (the FP64 oracle timed on the host
cores) prints one JSON line with the contract's keys, N > 1 ranks other than
rank 0 print nothing, and the flop / byte / traffic helpers agree with their
definitions (3 s^2 L + s^3 algorithmic flops per step, Gram and A^2 counted
once; 6 s L + 6 s^2 BF16 bytes; traffic only for the recorded kernel hash).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_flop_and_byte_counts():
    assert bench.algorithmic_flops([(768, 3072)], 1) == 3 * 768 ** 2 * 3072 + 768 ** 3
    assert bench.algorithmic_flops([(3072, 768)], 5) == 5 * (3 * 768 ** 2 * 3072 + 768 ** 3)
    assert bench.dense_equiv_flops([(100, 40)], 2) == 2 * (4 * 40 ** 2 * 100 + 2 * 40 ** 3)
    assert bench.algorithmic_bytes_bf16([(64, 256)], 1) == 6 * 64 * 256 + 6 * 64 * 64
    # the GPT-2-small step: 217 GFLOP per polynomial step
    f = bench.algorithmic_flops([(768, 2304), (768, 768), (768, 3072), (3072, 768)] * 12, 1)
    assert abs(f - 2.174e11) < 1e9


def test_traffic_only_for_the_recorded_kernel_source():
    h = bench.kernel_source_hash("umma_step")
    assert len(h) == 16 and h == bench.kernel_source_hash("umma_step")
    with open(os.path.join(ROOT, "profiles", "traffic.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    for wl, kern, hsh, nbytes in rows:
        got = bench.committed_traffic(wl, kern)
        assert got == (float(nbytes) if hsh == bench.kernel_source_hash(kern) else None)
    assert bench.committed_traffic("no_such_workload", "umma_step") is None


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    p = _run(["--impl", "reference", "--steps", "2", "--warmup", "3", "--workload", "plain_small"])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] >= 3
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["config"]["workload"]


def test_reference_arm_other_ranks_print_nothing():
    p = _run(["--impl", "reference", "--steps", "1", "--warmup", "3", "--workload", "plain_small"],
             env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


@pytest.mark.parametrize("argv", [["--steps", "0"], ["--warmup", "1", "--steps", "2"]])
def test_timing_rules_enforced(argv):
    """K >= 1 timed steps and W >= 3 warm-up steps (a smaller W is raised to 3)."""
    p = _run(["--impl", "reference", "--workload", "plain_small"] + argv)
    if "--steps" in argv and argv[argv.index("--steps") + 1] == "0":
        assert p.returncode == 2 and "--steps must be >= 1" in p.stderr
    else:
        assert p.returncode == 0, p.stderr[-2000:]
        assert json.loads(p.stdout.strip().splitlines()[-1])["warmup"] >= 3


def test_roofline_line():
    """The dominant kernel's roofline from a traced launch list: the fused
    step kernel against the BF16 peaks (burst and sustained), a phase kernel
    with its own flops, the FP32 path against the derived SIMT roof, and a
    memory-bound kernel against HBM."""
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1600.0, "sm_max_mhz": 2000.0,
             "source": "measured"}
    shapes = [(768, 3072), (3072, 768)]
    fs = bench.algorithmic_flops(shapes, 1)
    r = bench.roofline_line({"prepare": (5, 0.5), "umma_step": (25, 25 * 0.25)}, shapes, "bf16", fs, 1e8,
                            "no_such_workload", peaks)
    assert r["kernel"] == "umma_step" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - fs / 0.25e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 2000.0) < 1e-12 and abs(r["frac_sustained"] - r["achieved"] / 1600.0) < 1e-12
    assert r["traffic"] is None and abs(r["share_of_step"] - 6.25 / 6.75) < 1e-12
    r = bench.roofline_line({"umma_update": (10, 1.0), "umma_gram": (10, 0.5)}, shapes, "bf16", fs, 1e8, "x", peaks)
    assert r["kernel"] == "umma_update"
    assert abs(r["achieved"] - 2 * 2.0 * 768 ** 2 * 3072 / 0.1e-3 / 1e12) < 1e-6
    r = bench.roofline_line({"simt_update": (10, 1.0)}, shapes, "fp32", fs, 1e8, "x", peaks)
    assert r["bound"] == "alu" and abs(r["peak"] - 152 * 128 * 2 * 2000e6 / 1e12) < 1e-9 and "frac_sustained" not in r
    r = bench.roofline_line({"prepare": (4, 2.0)}, shapes, "bf16", fs, 1e8, "x", peaks)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and abs(r["achieved"] - 2e8 / 0.5e-3 / 1e9) < 1e-9


def test_rank_sets_share_shapes_not_values():
    """The multi-GPU weak-scaling run gives every rank its own set: the
    single-GPU set's shapes and distributions, other seeds."""
    a = bench.CPU_WORKLOADS["gpt2_small"]()
    b = bench.RANK_WORKLOADS["gpt2_small"](1)
    assert a.shapes == b.shapes and a.T == b.T and a.l == b.l
    assert not np.array_equal(a.matrices[0], b.matrices[0])
    assert abs(np.linalg.norm(b.matrices[0]) - np.linalg.norm(a.matrices[0])) < 1e-9
