"""Host logic of the benchmark and the binding (no GPU): the roofline's
per-entry work and the peak it divides by for each precision, the reported
traffic, and the precision constants against the C header."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1700.0}


def test_split_forms_count_three_products():
    # d = 64, t = 16: 2 (d + t) = 160 per product
    assert bench.tensor_flops_per_entry("split_f16", 64, 16) == 480.0
    assert bench.tensor_flops_per_entry("split_tf32", 64, 16) == 480.0
    assert bench.tensor_flops_per_entry("tf32", 64, 16) == 160.0


def test_roofline_is_algorithmic_work_over_sustained_peak():
    # N = 2^20, d = 64, t = 16: 2 N^2 (d + t) = 1.759e14 flops per product
    n, ms = 1 << 20, 500.0
    f16 = bench.roofline("split_f16", 64, 16, n, ms, float(n) ** 2, 2070.0, PEAKS, "test")
    tf32 = bench.roofline("split_tf32", 64, 16, n, ms, float(n) ** 2, 2070.0, PEAKS, "test")
    alg = 2.0 * n * n * 80 / 0.5 / 1e12
    assert f16["bound"] == tf32["bound"] == "tensor"
    assert f16["achieved"] == pytest.approx(alg)
    assert f16["peak"] == pytest.approx(1700.0)                 # FP16 = BF16 sustained
    assert tf32["peak"] == pytest.approx(1700.0 * 1.1 / 2.25)
    assert f16["frac"] == pytest.approx(alg / 1700.0)
    # the tensor pipe's own work (3 products per split form) is reported apart
    assert f16["pipe_tflops"] == pytest.approx(480.0 * n * n / 0.5 / 1e12)


def test_sfu_bound_counts_evaluated_entries():
    n = 1 << 20
    full = bench.roofline("split_f16", 64, 16, n, 100.0, float(n) ** 2, 2000.0, PEAKS, "test")
    half = bench.roofline("split_f16", 64, 16, n, 100.0, float(n) ** 2 / 2, 2000.0, PEAKS, "test")
    per = 1.0 / 30 + 1.0 / 15
    bound_ms = float(n) ** 2 * per / (152 * 2000.0e6) * 1e3
    assert full["sfu"]["bound_ms"] == pytest.approx(bound_ms)
    assert half["sfu"]["bound_ms"] == pytest.approx(bound_ms / 2)
    assert full["sfu"]["frac"] == pytest.approx(bound_ms / 100.0)


def test_roofline_fp32_is_alu_bound():
    n = 65536
    r = bench.roofline("fp32", 32, 32, n, 20.0, float(n) ** 2, 2000.0, PEAKS, "test")
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 128 * 2000.0e6 / 1e12)
    assert r["achieved"] == pytest.approx(2.0 * n * n * 64 / 0.02 / 1e12)


def test_traffic_is_the_captured_launch():
    # the DRAM bytes of one captured launch of the current kernel (read +
    # write); no entry for forms whose kernels changed since a capture
    assert bench.KMV_DRAM_BYTES[("gp1m", "split_f16")] == 3344414208 + 668886528
    for key, v in bench.KMV_DRAM_BYTES.items():
        assert key[0] in bench.WORKLOADS and key[1] in ("split_f16", "split_tf32", "fp32")
        assert isinstance(v, int) and v > 0
    assert bench.KMV_DRAM_BYTES.get(("gp1m", "split_tf32")) is None


def test_precision_constants_match_header():
    src = open(os.path.join(ROOT, "include", "gp.h")).read()
    enum = dict((m.group(1), int(m.group(2)))
                for m in re.finditer(r"\b(GP_(?:FP32_PLAIN|FP32_SPLIT_TF32|FP32_SPLIT_F16|TF32))\s*=\s*(\d+)", src))
    from paper_2109_09817_gb300 import _lib
    assert enum == {"GP_FP32_PLAIN": _lib.GP_FP32_PLAIN, "GP_FP32_SPLIT_TF32": _lib.GP_FP32_SPLIT_TF32,
                    "GP_FP32_SPLIT_F16": _lib.GP_FP32_SPLIT_F16, "GP_TF32": _lib.GP_TF32}
    assert "GP_BF16" not in src


def test_bench_default_is_split_f16():
    args = bench.parse([])
    assert args.precision == "split_f16" and args.warmup >= 3 and args.gpus == 1
    assert args.stop == "true" and args.workload == "gp1m"
