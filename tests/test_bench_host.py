"""The benchmark's algorithmic work counts (the roofline numerators), against their
closed forms for regular codes, and its command line.  CPU only."""
import subprocess
import sys
import os

import numpy as np
import pytest

from paper_2508_03567_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("name", ["gf4_n48_dv2_dc4", "gf64_n576_dv2_dc4", "gf32_n600_dv3_dc6",
                                  "gf256_n128_dv2_dc8"])
def test_minmax_pairs_per_frame_iteration(name):
    """3(d_c - 2) q^2 min-max pairs per check (forward, backward and middle convolutions)."""
    code = I.workload_code(name)
    w = I.WORKLOADS[name]
    assert bench.pairs_per_frame_iter(code) == code.m * 3 * (w["dc"] - 2) * code.q ** 2


@pytest.mark.parametrize("name", ["gf4_n48_dv2_dc4", "gf64_n576_dv2_dc4", "gf32_n600_dv3_dc6"])
def test_fftspa_float_operations_per_frame_iteration(name):
    """E q (2 log2 q + d_c + d_v + 2) for a regular code (Table 1's FFT-SPA rows without loop
    control); GF(64) (2,4) N=576: 1,474,560."""
    code = I.workload_code(name)
    w = I.WORKLOADS[name]
    e = code.nnz
    assert bench.fft_flops_per_frame_iter(code) == e * code.q * (2 * code.p + w["dc"] + w["dv"] + 2)
    if name == "gf64_n576_dv2_dc4":
        assert bench.fft_flops_per_frame_iter(code) == 1474560


def test_irregular_counts_sum_over_rows_and_columns():
    h = np.zeros((3, 6), np.int64)
    h[0, [0, 1, 2]] = 1
    h[1, [2, 3, 4, 5]] = 2
    h[2, [0, 5]] = 3
    code = I.code_from_dense(h, 4, I.PRIMITIVE_POLY[4])
    assert bench.pairs_per_frame_iter(code) == (3 * 1 + 3 * 2 + 0) * 16
    d = np.array([3, 4, 2])
    v = np.array([2, 1, 2, 1, 1, 2])
    want = int((2 * d * 4 * 2 + d * (d - 1) * 4 + d * 4).sum() + (v * (v - 1) * 4 + 3 * v * 4).sum())
    assert bench.fft_flops_per_frame_iter(code) == want


def test_command_line_lists_every_workload():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True,
                         text=True, check=True).stdout
    for mode in ("gf64", "mixed", "serving", "width", "fftspa", "schedule"):
        assert mode in out
