"""GPU parity of the pruned check-node convolutions (tuning variants 4 and 5)
and the work counter.

The pruned convolution folds in only the entries of one side that are at most
a bound T >= max_x C(x) and finds T in phases; its outputs must equal the
oracle's bit for bit on every input, including those that make the bound
search take its rare paths: every value equal (C is constant, the first phase
already covers it), only 0 and 255 (bounds jump), all zeros, ties, and
messages whose first phase folds in nothing."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2508_03567_gb300 import binding, inputs as I

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def assert_same(got, want, ctx=""):
    for n, g, w in zip(("symbols", "iterations", "ok"), got, want):
        if not np.array_equal(g, w):
            bad = np.nonzero((g != w).reshape(g.shape[0], -1).any(1))[0]
            raise AssertionError(f"{ctx}: {n} differ in {bad.size} frames, first {bad[:8].tolist()}")


def decode_with(dec, g, mi, early):
    out = [t.cpu().numpy() for t in dec.decode(torch.as_tensor(g).cuda(), mi, early)]
    torch.cuda.synchronize()
    return out


def adversarial(kind, f, n, q, seed):
    rng = np.random.default_rng(seed)
    if kind == "all_equal":
        return np.full((f, n, q), 9, np.uint8)
    if kind == "saturated":
        return rng.choice(np.array([0, 255], np.uint8), (f, n, q))
    if kind == "random_u8":
        return rng.integers(0, 256, (f, n, q)).astype(np.uint8)
    if kind == "zeros":
        return np.zeros((f, n, q), np.uint8)
    if kind == "ties_small":
        return rng.integers(0, 2, (f, n, q)).astype(np.uint8)
    if kind == "one_small":      # one entry 0 per row, the rest 200..255: large maxima, sparse small sets
        g = rng.integers(200, 256, (f, n, q)).astype(np.uint8)
        g[np.arange(f)[:, None], np.arange(n)[None, :], rng.integers(0, q, (f, n))] = 0
        return g
    raise ValueError(kind)


PR_CODES = [(64, 48, 2, 4, (4,)), (128, 72, 2, 6, (4, 5)), (256, 32, 2, 4, (4, 5)), (256, 64, 2, 8, (4,))]
KINDS = ["all_equal", "saturated", "random_u8", "zeros", "ties_small", "one_small"]


@pytest.mark.parametrize("q,n,dv,dc,variants", PR_CODES)
def test_pruned_variants_match_the_oracle(q, n, dv, dc, variants):
    code = I.make_regular_code(q, n, dv, dc, seed=13 * q + n)
    dec = binding.Decoder.from_code(code)
    cases = [("channel", I.make_batch(code, eb, 17 + q, 12).gamma.numpy(), mi, early)
             for eb, mi, early in ((1.0, 9, 1), (2.5, 6, 0))]
    cases += [(k, adversarial(k, 5, code.n, q, q + i), 5, 1) for i, k in enumerate(KINDS)]
    for v in variants:
        for fpb in (1, 2):
            dec.set_tuning(v, fpb)
            assert dec.tuning() == (v, fpb)
            for name, g, mi, early in cases:
                assert_same(decode_with(dec, g, mi, early), oracle.decode(code, g, mi, early, threads=THREADS),
                            f"q={q} variant {v} fpb {fpb} {name}")


def test_pruned_and_dense_codes_in_one_mixed_batch():
    """The all-field kernel prunes the GF(128)/GF(256) jobs whose variant has bit 2 and keeps the
    dense convolution for the others; every job equals the oracle."""
    specs = []
    for k, (name, v, frames) in enumerate((("gf256_n128_dv2_dc8", 4, 9), ("gf256_n384_dv2_dc6", 0, 3),
                                           ("gf64_n576_dv2_dc4", 4, 4), ("gf16_n1024_dv2_dc4", 1, 7))):
        w = I.WORKLOADS[name]
        code = I.workload_code(name)
        dec = binding.Decoder.from_code(code)
        dec.set_tuning(v, 1)
        g = I.make_batch(code, 2.0, 808 + k, frames).gamma.numpy()
        gd = torch.as_tensor(g).cuda().contiguous()
        out = (torch.empty((frames, code.n), dtype=torch.uint8, device="cuda"),
               torch.empty((frames,), dtype=torch.int32, device="cuda"),
               torch.empty((frames,), dtype=torch.uint8, device="cuda"))
        specs.append((code, dec, g, gd, out, w["max_iters"], w["early_stop"]))
    jobs = [(d.handle, gd, g.shape[0], mi, es, *out) for code, d, g, gd, out, mi, es in specs]
    ws = torch.empty(binding.nbldpc_decode_batch_workspace_size(jobs), dtype=torch.uint8, device="cuda")
    binding.nbldpc_decode_batch(jobs, ws)
    torch.cuda.synchronize()
    for code, d, g, gd, out, mi, es in specs:
        assert_same([t.cpu().numpy() for t in out], oracle.decode(code, g, mi, es, threads=THREADS),
                    f"batch q={code.q}")


def test_unsupported_pruned_tunings_are_rejected():
    def status(code, v):
        dec = binding.Decoder.from_code(code)
        try:
            dec.set_tuning(v, 1)
            return binding.NBLDPC_OK
        except binding.NbldpcError as e:
            return e.status
    q16 = I.workload_code("gf16_n1024_dv2_dc4")
    q64 = I.workload_code("gf64_n576_dv2_dc4")
    q256 = I.workload_code("gf256_n128_dv2_dc8")
    assert status(q16, 4) == binding.NBLDPC_ERR_UNSUPPORTED      # 16-lane groups
    assert status(q64, 5) == binding.NBLDPC_ERR_UNSUPPORTED      # GF(64) layout 1: 16-lane groups
    assert status(q256, 6) == binding.NBLDPC_ERR_UNSUPPORTED     # with resident messages
    assert status(q256, 8) == binding.NBLDPC_ERR_ARG
    dec = binding.Decoder.from_code(q256)
    assert dec.tuning()[0] == 4                                   # the default of GF(256)
    dec.set_message_bits(16)                                      # 16-bit messages keep the layout bit only
    assert dec.tuning()[0] == 0
    with pytest.raises(binding.NbldpcError):
        dec.set_tuning(4, 1)


def dense_pairs(code, iters):
    d = np.diff(code.row_ptr)
    return int(np.asarray(iters, np.int64).sum()) * int((3 * np.maximum(d - 2, 0)).sum()) * code.q ** 2


@pytest.mark.parametrize("name,variant,fpb", [("gf4_n48_dv2_dc4", 2, 1), ("gf4_n48_dv2_dc4", 2, 8),
                                              ("gf4_n48_dv2_dc4", 0, 1), ("gf16_n1024_dv2_dc4", 1, 1),
                                              ("gf64_n576_dv2_dc4", 3, 1), ("gf256_n128_dv2_dc8", 0, 1)])
def test_work_counter_of_dense_convolutions_is_the_schedule_count(name, variant, fpb):
    """Dense convolutions visit q^2 pairs each, 3(d_c - 2) per check and iteration (the GF(4)
    register form, the GF(4) one-warp form at 8 frames per block, and the group form alike)."""
    w = I.WORKLOADS[name]
    code = I.workload_code(name)
    dec = binding.Decoder.from_code(code)
    dec.set_tuning(variant, fpb)
    g = I.make_batch(code, w["ebn0"][0], 909, 40).gamma.cuda()
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    binding.nbldpc_code_set_work_counter(dec.handle, cnt)
    s, its, ok = dec.decode(g, w["max_iters"], w["early_stop"])
    torch.cuda.synchronize()
    assert int(cnt.item()) == dense_pairs(code, its.cpu().numpy())
    binding.nbldpc_code_set_work_counter(dec.handle, None)        # off: the counter stays
    dec.decode(g, w["max_iters"], w["early_stop"])
    torch.cuda.synchronize()
    assert int(cnt.item()) == dense_pairs(code, its.cpu().numpy())


def test_work_counter_of_pruned_convolutions():
    """A pruned convolution visits q pairs per entry it folds in: the count is a multiple of q, far
    below the dense count, the same on a repeated decode, and the outputs are those of the dense
    variant."""
    name = "gf256_n384_dv2_dc6"
    w = I.WORKLOADS[name]
    code = I.workload_code(name)
    dec = binding.Decoder.from_code(code)
    g = I.make_batch(code, 2.5, 910, 64).gamma.cuda()
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    binding.nbldpc_code_set_work_counter(dec.handle, cnt)
    counts, outs = [], []
    for v in (4, 4, 0):
        dec.set_tuning(v, 1)
        cnt.zero_()
        outs.append([t.cpu().numpy() for t in dec.decode(g, w["max_iters"], w["early_stop"])])
        torch.cuda.synchronize()
        counts.append(int(cnt.item()))
    dense = dense_pairs(code, outs[2][1])
    assert counts[2] == dense
    assert counts[0] == counts[1] and counts[0] % code.q == 0
    assert 0 < counts[0] < dense // 4
    assert_same(outs[0], outs[2], "pruned vs dense")
