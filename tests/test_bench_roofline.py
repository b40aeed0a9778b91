"""bench.py's roofline record of the shifted SpMM, checked against byte and flop counts
worked out by hand for a small pencil (no GPU).

Pencil: n = 100 rows, 2,700 pattern entries, 900 nonzeros of B; k = 4 columns, m = 8
poles, so W = 32 complex columns.
  bytes, FP32 state (8 B per complex entry, 4 B per value): 5 * 8 * 100 * 32 + 2,700 * (4 + 2 * 4)
        = 128,000 + 32,400 = 160,400
  bytes, FP64 state (16 B, 8 B values): 5 * 16 * 100 * 32 + 2,700 * (4 + 2 * 8) = 310,000
  flops over the pattern: 8 * 2,700 * 32 + 32 * 100 * 32 = 691,200 + 102,400 = 793,600
  flops executed with B-diagonal records (A's entries + B's nonzeros): (4 * 2,700 + 4 * 900) * 32
        + 102,400 = 563,200
FP32 at 3.5 flop/B is below GB300's FP32-to-HBM balance (about 12 flop/B), so HBM bounds it;
FP64 at 2.56 flop/B is above the FP64 balance (about 0.19 flop/B), so the FP64 pipe does.
"""
import types

import numpy as np
import pytest

import bench


def _pencil():
    valB = np.zeros(2700)
    valB[:900] = 1.0
    return types.SimpleNamespace(n=100, nnz=2700, valB=valB)


def test_fp32_b_diagonal_is_hbm_bound():
    hbm, _ = bench.measured_hbm_gbs()
    r = bench.spmm_roofline(_pencil(), m=8, k=4, precision=1, spmm_ms=1e-3, traffic=None, bdiag=True)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None
    assert r["bytes_per_launch"] == 160_400
    assert r["flops_pattern_per_launch"] == 793_600
    assert r["flops_per_launch"] == 563_200
    assert r["achieved"] == pytest.approx(160.4)  # 160,400 B in 1 us
    assert r["peak"] == hbm and r["frac"] == pytest.approx(160.4 / hbm)
    assert r["b_diagonal_records"] is True


def test_general_records_count_every_pattern_product():
    r = bench.spmm_roofline(_pencil(), m=8, k=4, precision=1, spmm_ms=1e-3, traffic=7.0e5, bdiag=False)
    assert r["flops_per_launch"] == r["flops_pattern_per_launch"] == 793_600
    assert r["traffic"] == 7.0e5


def test_fp64_is_alu_bound():
    r = bench.spmm_roofline(_pencil(), m=8, k=4, precision=0, spmm_ms=1e-3, traffic=None)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["bytes_per_launch"] == 310_000
    assert r["achieved"] == pytest.approx(0.7936)  # 793,600 flops in 1 us
    assert r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS)
    assert r["hbm_gbs_algorithmic"] == pytest.approx(310.0)
