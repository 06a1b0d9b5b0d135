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


# ---- Table 1 of the paper (operation counts per iteration; memory transactions left out)
# Each row restated as (additions, multiplications, divisions, comparisons) for a regular
# code with M checks of degree dc, N variables of degree dv and field order g.

def _table1_minmax(M, N, dc, dv, g):
    lc_c = M + M * dc + M * dc * g          # loop control of the per-check passes
    lc_v = N + N * dv + N * dv * g
    return {
        "fb_first_lc": (lc_c, 0, 0, lc_c),
        "fb_first": (0, 0, 0, M * dc * g),
        "fb_rest_lc": (M * (dc - 1) * g * g, 0, 0, M * (dc - 1) * g * g),
        "fb_rest": (2 * M * (dc - 1) * g * g, 0, 0, 2 * M * (dc - 1) * g * g + 2 * M * (dc - 1) * g),
        "beta_ends_lc": (lc_c, 0, 0, lc_c),
        "beta_ends": (0, 0, 0, 2 * M * dc * g),
        "beta_rest_lc": (M * (dc - 2) * g * g, 0, 0, M * (dc - 2) * g * g),
        "beta_rest": (M * (dc - 2) * g * g, 0, 0, M * (dc - 2) * g * g + M * (dc - 2) * g),
        "vnp_lc": (lc_v, 0, 0, lc_v),
        "vnp": (N * dv * (dv - 1) * g + 2 * N * dv * g, 0, 0, N * dv * g),
    }


def _table1_fftspa(M, N, dc, dv, g, lg):
    lc_c = M + M * dc + M * dc * g
    lc_v = N + N * dv + N * dv * g
    e = M * dc
    return {
        "perm_lc": (lc_v, 0, 0, lc_v),
        "perm": (0, 0, 0, 0),
        "cnp_lc": (lc_c, 0, 0, lc_c),
        "fft": (e * g * lg, e * g * lg, 0, 0),
        "product": (e * (dc - 1) * g, e * (dc - 1) * g, 0, 0),
        "ifft": (e * g * lg, e * g * lg, e * g, 0),
        "deperm_lc": (lc_c, 0, 0, lc_c),
        "deperm": (0, 0, 0, 0),
        "vnp_lc": (lc_v, 0, 0, lc_v),
        "vnp": (N * dv * g, N * dv * (dv - 1) * g + N * dv * g, N * dv * g, 0),
    }


SHAPES = [(24, 48, 4, 2, 4, 2), (288, 576, 4, 2, 64, 6), (300, 600, 6, 3, 32, 5), (32, 128, 8, 2, 256, 8),
          (7, 21, 9, 3, 8, 3)]


@pytest.mark.parametrize("M,N,dc,dv,g,lg", SHAPES)
def test_table1_rows_sum_to_the_printed_totals(M, N, dc, dv, g, lg):
    """Sec. 3's closed forms for the total operation counts (memory transactions excluded) are
    the sums of Table 1's rows, for both decoders."""
    mm = sum(sum(r) for r in _table1_minmax(M, N, dc, dv, g).values())
    assert mm == (4 * M + 4 * M * dc - 4 * M * g - 14 * M * g * g + 10 * M * dc * g + 10 * M * dc * g * g
                  + 2 * N + 2 * N * dv + 4 * N * dv * g + N * dv * dv * g)
    ff = sum(sum(r) for r in _table1_fftspa(M, N, dc, dv, g, lg).values())
    assert ff == (4 * M + 4 * M * dc + 3 * M * dc * g + 2 * M * dc * dc * g + 4 * M * dc * g * lg
                  + 4 * N + 4 * N * dv + 6 * N * dv * g + N * dv * dv * g)


@pytest.mark.parametrize("name", ["gf4_n48_dv2_dc4", "gf64_n576_dv2_dc4", "gf32_n600_dv3_dc6",
                                  "gf256_n128_dv2_dc8"])
def test_convolution_counts_against_table1(name):
    """Table 1 lists one GF addition (the XOR of the two indices) per min-max pair of the
    forward/backward and middle convolutions: M(3dc - 4) g^2 pairs, the count of the Table 1
    schedule; the minimal schedule drops the two convolutions whose outputs no message uses."""
    code = I.workload_code(name)
    w = I.WORKLOADS[name]
    rows = _table1_minmax(code.m, code.n, w["dc"], w["dv"], code.q)
    t1_pairs = rows["fb_rest"][0] + rows["beta_rest"][0]
    assert bench.convolutions_per_frame_iter(code, table1=True) * code.q ** 2 == t1_pairs
    assert bench.convolutions_per_frame_iter(code) * code.q ** 2 == t1_pairs - 2 * code.m * code.q ** 2
    assert bench.pairs_per_frame_iter(code) == t1_pairs - 2 * code.m * code.q ** 2


@pytest.mark.parametrize("name", ["gf4_n48_dv2_dc4", "gf64_n576_dv2_dc4", "gf32_n600_dv3_dc6",
                                  "gf256_n128_dv2_dc8"])
def test_fftspa_count_against_table1(name):
    """The float-operation count is Table 1's FFT-SPA rows without loop control, less the
    transforms' multiplications (+-1 factors) and the additions beside the check-node products."""
    code = I.workload_code(name)
    w = I.WORKLOADS[name]
    rows = _table1_fftspa(code.m, code.n, w["dc"], w["dv"], code.q, code.p)
    no_lc = sum(sum(r) for k, r in rows.items() if not k.endswith("_lc"))
    dropped = rows["fft"][1] + rows["ifft"][1] + rows["product"][0]
    assert bench.fft_flops_per_frame_iter(code) == no_lc - dropped


@pytest.mark.parametrize("q,d", [(4, 2), (4, 4), (8, 5), (16, 6), (64, 4)])
def test_oracle_visits_the_pairs_the_counts_assume(q, d):
    """The oracle's check update, instrumented, visits (d - 2) q^2 pairs in each of its forward,
    backward and beta remaining-edge blocks: the 3(d - 2) q^2 per check of the roofline numerator.
    Table 1 lists (d - 1) q^2 for each of F and B (its F_{d-1} and B_0 feed no message) and
    (d - 2) q^2 for beta."""
    import oracle
    rng = np.random.default_rng(q * 100 + d)
    h = rng.integers(1, q, d)
    alpha = rng.integers(0, 64, (d, q))
    beta, pairs = oracle.check_update_pairs(q, I.PRIMITIVE_POLY[q], h, alpha)
    assert np.array_equal(beta, oracle.check_update(q, I.PRIMITIVE_POLY[q], h, alpha))
    assert list(pairs) == [(d - 2) * q * q] * 3
    code = I.code_from_dense(np.array([h]), q, I.PRIMITIVE_POLY[q])
    assert bench.pairs_per_frame_iter(code) == int(pairs.sum())
    rows = _table1_minmax(1, d, d, 1, q)
    assert rows["fb_rest"][0] == pairs[0] + pairs[1] + 2 * q * q
    assert rows["beta_rest"][0] == pairs[2]


def test_code_hash_ignores_comments_and_layout_only():
    """The profile fingerprint: comments and whitespace do not count, code and literals do."""
    a = "int f(int x) {  // twice\n  return 2 * x; /* doubled */ }\n"
    b = "/* header */\nint f(int x) {\n\n  return 2 * x;\n}"
    c = "int f(int x) { return 3 * x; }"
    assert bench.strip_comments(a) == bench.strip_comments(b) == "int f(int x) { return 2 * x; }"
    assert bench.strip_comments(c) != bench.strip_comments(a)
    assert bench.strip_comments('s = "a // b /* c */";') == 's = "a // b /* c */";'
    assert bench.strip_comments("char q = '\\''; // x") == "char q = '\\'';"
    assert len(bench.kernel_code_hash("fftspa_kernels.cuh")) == 16


def test_command_line_lists_every_workload():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True,
                         text=True, check=True).stdout
    for mode in ("gf64", "mixed", "serving", "width", "fftspa", "schedule"):
        assert mode in out


def test_measured_peak_and_issue_bound_arithmetic(monkeypatch):
    """The roofline denominators: the probe's best pairs/clk/SM x 2 u16 ops x SMs x the maximum
    SM clock, beside the issue-bound 256 ops/clk/SM; frac and frac_issue_bound divide by them."""
    monkeypatch.setattr(bench, "sm_count", lambda dev: 152)
    monkeypatch.setattr(bench, "sm_max_mhz", lambda: (2070.0, "measured"))
    meas = {"pairs_per_clk_sm": 88.0, "best_form": "fma_3_8"}
    peak, kind, issue = bench.alu_peaks(meas, None)
    assert peak == pytest.approx(152 * 2 * 88.0 * 2070e6 / 1e9)
    assert issue == pytest.approx(152 * 256 * 2070e6 / 1e9)
    assert "measured" in kind and "fma_3_8" in kind
    peak0, kind0, issue0 = bench.alu_peaks(None, None)
    assert peak0 == issue0 and kind0.startswith("derived")
    r = bench.roofline_alu(0.5 * peak, peak, kind, issue)
    assert r["frac"] == pytest.approx(0.5) and r["frac_issue_bound"] == pytest.approx(0.5 * peak / issue)
    assert r["bound"] == "alu" and r["unit"] == "Gop/s"


def test_small_workloads_rotate_through_more_than_l2():
    """A step whose inputs fit L2 rotates through distinct batches totalling more than L2;
    a step larger than L2 is decoded as it is."""
    gf4 = 1000 * 48 * 4                       # GF(4) N=48, 1000 frames
    n = bench.batch_pool(gf4)
    assert n > 1 and n * gf4 > bench.L2_BYTES and (n - 1) * gf4 < 2 * bench.L2_BYTES
    assert bench.batch_pool(196608 * 576 * 64) == 1   # the GF(64) step
    assert bench.batch_pool(16384 * 384 * 256) == 1   # GF(256) N=384, 16384 frames


def test_hbm_roof_beside_the_alu_roof():
    """The roofline object also carries the HBM fraction: algorithmic bytes (reliabilities in,
    outputs out) per second against the copy bandwidth; for the GF(64) step it is tiny, so the ALU
    roof binds."""
    code = I.workload_code("gf64_n576_dv2_dc4")
    assert bench.algorithmic_bytes_per_frame(code) == 576 * 64 + 576 + 5 == 37445
    r = bench.roofline_alu(40e3, 55e3, "measured", 80e3, None, 196608 * 37445 / 0.7)
    gbs, _ = bench.hbm_peak_gbs()
    assert r["hbm"]["unit"] == "GB/s" and r["hbm"]["frac"] == pytest.approx(196608 * 37445 / 0.7 / 1e9 / gbs)
    assert r["hbm"]["frac"] < 0.01 < r["frac"]


def test_pruned_work_is_reported_beside_the_dense_count():
    """The roofline counts the pairs the kernel visited; a pruned decode also reports the rate its
    time gives the paper's dense count (which may exceed the peak), a dense one does not."""
    r = bench.roofline_alu(30e3, 55e3, "measured", 80e3, dense=120e3)
    assert r["frac"] == pytest.approx(30 / 55) and r["work"].startswith("executed")
    assert r["dense_equivalent"]["frac"] == pytest.approx(120 / 55)
    r = bench.roofline_alu(30e3, 55e3, "measured", 80e3, dense=30e3)
    assert "dense_equivalent" not in r and "work" not in r
