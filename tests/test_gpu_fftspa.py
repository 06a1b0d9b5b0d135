"""GPU parity of the FFT-SPA decoder (Alg. 1, float) against the float64
oracle, through the C ABI.

Decisions (symbols, iterations, ok flags) must equal the oracle's; a frame
may differ only where the oracle itself sits on a near-tie (top two
a-posteriori values within 1e-4), which float rounding can flip.

The a-posteriori vectors after k iterations must agree element by element
within app_tol(code, k): with unit roundoff u = 2^-24, one iteration takes
every a-posteriori component through at most L = 3 log2(q) + d_c + d_v + 4
rounded operations on values bounded by 1 (two radix-2 transforms of log2(q)
stages, d_c - 1 products and the 1/q scale at the check node; d_v products,
a log2(q)-deep sum, a reciprocal and a multiply at the variable node), each
off by at most u.  The normalization divides by sums below 1, which amplifies
absolute errors; the bound allows a factor 2^8 for it and adds the k
iterations linearly, so it is checked for k <= 2 only (beyond that the
decisions are compared)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_03567_gb300 import binding, inputs as I

pytestmark = pytest.mark.gpu
THREADS = 16
U = 2.0 ** -24


def app_tol(code, k):
    p = code.p
    dc = int(np.diff(code.row_ptr).max())
    dv = int(np.bincount(code.col_idx).max())
    return 256.0 * (3 * p + dc + dv + 4) * max(k, 1) * U


def near_tie(app_row_set):
    """Per frame: the smallest gap between the two largest a-posteriori values over its symbols."""
    s = np.sort(app_row_set, -1)
    return (s[..., -1] - s[..., -2]).min(-1)


def assert_decisions(code, got, want, app_want, what):
    sym, its, ok = (t.cpu().numpy() if torch.is_tensor(t) else t for t in got)
    diff = (sym != want[0]).any(1) | (its != want[1]) | (ok != want[2])
    if diff.any():
        gaps = near_tie(app_want[diff])
        assert np.all(gaps < 1e-4), f"{what}: {int(diff.sum())} frames differ, oracle gaps {gaps[:8]}"
    assert diff.mean() <= 0.02, f"{what}: {int(diff.sum())} of {diff.size} frames differ"


def irregular_code(q, seed, dmax=8):
    """Rows of degree 2..dmax, columns of degree >= 1, random coefficients (degrees stay within the limits)."""
    rng = np.random.default_rng(seed)
    n, m = (70, 30) if dmax <= 8 else (260, 30)
    h = np.zeros((m, n), np.int64)
    for r in range(m):
        d = int(rng.integers(2, dmax + 1))
        cols = rng.choice(n, d, replace=False)
        h[r, cols] = rng.integers(1, q, d)
    for c in range(n):
        if not h[:, c].any():
            rows = [r for r in range(m) if (h[r] != 0).sum() < dmax]
            h[int(rng.choice(rows)), c] = int(rng.integers(1, q))
    return I.code_from_dense(h, q, I.PRIMITIVE_POLY[q])


CODES = [
    ("gf4_n48_dv2_dc4", None, 3.0, 48),
    ("gf64_n576_dv2_dc4", None, 2.0, 24),
    ("gf256_n128_dv2_dc8", None, 2.0, 12),
    ("gf32_n600_dv3_dc6", None, 2.0, 24),
    ("gf16_n1024_dv2_dc4", None, 2.0, 12),
    ("q2_n60_dv3_dc6", (2, 60, 3, 6), 1.0, 48),
    ("q8_n64_dv2_dc4", (8, 64, 2, 4), 1.0, 48),
    ("q128_n96_dv2_dc4", (128, 96, 2, 4), 1.5, 12),
]


def code_of(name, shape):
    if shape is None:
        return I.workload_code(name)
    q, n, dv, dc = shape
    return I.make_regular_code(q, n, dv, dc, seed=31 * q + n)


@pytest.mark.parametrize("name,shape,eb,frames", CODES)
def test_app_within_the_derived_tolerance(name, shape, eb, frames):
    code = code_of(name, shape)
    p = I.make_batch(code, eb, 77, frames, prob=True).prob.numpy()
    dec = binding.Decoder.from_code(code)
    pd = torch.as_tensor(p).cuda()
    for k in (0, 1, 2):
        sym, its, ok, app = dec.fftspa_decode(pd, k, 0, want_app=True)
        ws, wi, wo, wapp = oracle.fftspa_decode(code, p, k, 0, threads=THREADS, want_app=True)
        err = np.abs(app.cpu().numpy().astype(np.float64) - wapp).max()
        assert err <= app_tol(code, k), f"{name} k={k}: max |dAPP| {err:.3e} > {app_tol(code, k):.3e}"
        assert_decisions(code, (sym, its, ok), (ws, wi, wo), wapp, f"{name} k={k}")


@pytest.mark.parametrize("name,shape,eb,frames", CODES)
def test_decisions_match_the_oracle(name, shape, eb, frames):
    code = code_of(name, shape)
    p = I.make_batch(code, eb, 91, frames, prob=True).prob.numpy()
    dec = binding.Decoder.from_code(code)
    pd = torch.as_tensor(p).cuda()
    for mi, early in ((25, 1), (8, 0)):
        got = dec.fftspa_decode(pd, mi, early)
        ws, wi, wo, wapp = oracle.fftspa_decode(code, p, mi, early, threads=THREADS, want_app=True)
        assert_decisions(code, got, (ws, wi, wo), wapp, f"{name} max_iters={mi} early={early}")
        # the a-posteriori output does not change the decisions
        got2 = dec.fftspa_decode(pd, mi, early, want_app=True)
        for a, b in zip(got, got2[:3]):
            assert torch.equal(a, b)


@pytest.mark.parametrize("q,dmax", [(4, 8), (16, 8), (64, 8), (256, 8), (2, 20), (8, 32), (32, 20), (64, 24)])
def test_irregular_code(q, dmax):
    """Check degrees up to 32 for q <= 64 (lane per edge), up to 8 for q = 256."""
    code = irregular_code(q, q + dmax, dmax)
    rng = np.random.default_rng(q + 1)
    w = rng.random((16, code.n, q)) ** 4
    hard = rng.integers(0, q, (16, code.n))
    w[np.arange(16)[:, None], np.arange(code.n)[None, :], hard] += 1.0
    p = (w / w.sum(-1, keepdims=True)).astype(np.float32)
    dec = binding.Decoder.from_code(code)
    for early in (0, 1):
        got = dec.fftspa_decode(torch.as_tensor(p).cuda(), 7, early)
        ws, wi, wo, wapp = oracle.fftspa_decode(code, p, 7, early, threads=THREADS, want_app=True)
        assert_decisions(code, got, (ws, wi, wo), wapp, f"irregular q={q} early={early}")


def test_degenerate_probabilities():
    """One-hot rows, all-zero rows (uniform fallback of the normalization) and uniform rows."""
    code = I.workload_code("gf16_n1024_dv2_dc4")
    rng = np.random.default_rng(5)
    p = I.make_batch(code, 2.0, 13, 8, prob=True).prob.numpy().copy()
    p[0] = 0.0                                         # all-zero frame
    p[1] = 1.0 / code.q                                # uniform frame
    idx = rng.integers(0, code.q, code.n)
    p[2] = 0.0
    p[2, np.arange(code.n), idx] = 1.0                 # one-hot, not a codeword in general
    p[3, ::7] = 0.0                                    # some all-zero symbols
    dec = binding.Decoder.from_code(code)
    for mi, early in ((6, 0), (20, 1)):
        got = dec.fftspa_decode(torch.as_tensor(p).cuda(), mi, early, want_app=True)
        ws, wi, wo, wapp = oracle.fftspa_decode(code, p, mi, early, threads=THREADS, want_app=True)
        assert_decisions(code, got[:3], (ws, wi, wo), wapp, f"degenerate max_iters={mi}")
        app = got[3].cpu().numpy()
        assert np.all(np.isfinite(app))
        np.testing.assert_allclose(app.sum(-1), 1.0, atol=1e-5)


def test_frame_counts_and_batch_independence():
    """0, 1, odd and more-than-resident frame counts; each frame's result is its own."""
    code = I.workload_code("gf4_n48_dv2_dc4")
    b = I.make_batch(code, 2.5, 31, 3001, prob=True)
    p = b.prob.numpy()
    dec = binding.Decoder.from_code(code)
    pd = torch.as_tensor(p).cuda()
    full = [t.cpu().numpy() for t in dec.fftspa_decode(pd, 15, 1)]
    ws, wi, wo, wapp = oracle.fftspa_decode(code, p, 15, 1, threads=THREADS, want_app=True)
    assert_decisions(code, full, (ws, wi, wo), wapp, "3001 frames")
    for lo, hi in ((0, 1), (5, 12), (1000, 1001), (17, 1200)):
        part = [t.cpu().numpy() for t in dec.fftspa_decode(pd[lo:hi].contiguous(), 15, 1)]
        for a, c in zip(part, full):
            assert np.array_equal(a, c[lo:hi])
    # zero frames queue nothing
    ws0 = dec.fftspa_workspace(1, "cuda")
    binding.nbldpc_fftspa_decode(dec.handle, pd, 0, 10, 1, None, None, None, None, ws0)


def test_noiseless_frames_decode_at_once():
    code = I.workload_code("gf64_n576_dv2_dc4")
    b = I.make_batch(code, 3.0, 17, 16, noiseless=True, prob=True)
    dec = binding.Decoder.from_code(code)
    sym, its, ok = (t.cpu().numpy() for t in dec.fftspa_decode(b.prob.cuda(), 10, 1))
    assert np.array_equal(sym.astype(np.int64), b.codewords.numpy())
    assert np.all(its == 0) and np.all(ok == 1)


def test_arguments_are_checked():
    code = I.workload_code("gf4_n48_dv2_dc4")
    dec = binding.Decoder.from_code(code)
    p = torch.full((4, code.n, code.q), 0.25, device="cuda")
    sym = torch.empty((4, code.n), dtype=torch.uint8, device="cuda")
    its = torch.empty(4, dtype=torch.int32, device="cuda")
    ok = torch.empty(4, dtype=torch.uint8, device="cuda")
    need = binding.nbldpc_fftspa_workspace_size(dec.handle, 4)
    ws = torch.empty(need + 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(binding.NbldpcError) as ei:        # workspace too small
        binding.nbldpc_fftspa_decode(dec.handle, p, 4, 5, 1, sym, its, ok, None, ws, need - 1)
    assert ei.value.status == binding.NBLDPC_ERR_ARG
    with pytest.raises(binding.NbldpcError) as ei:        # probabilities not 16-byte aligned
        binding.nbldpc_fftspa_decode(dec.handle, p.view(-1)[1:].data_ptr(), 3, 5, 1, sym, its, ok, None, ws)
    assert ei.value.status == binding.NBLDPC_ERR_ARG
    with pytest.raises(binding.NbldpcError) as ei:        # negative iteration count
        binding.nbldpc_fftspa_decode(dec.handle, p, 4, -1, 1, sym, its, ok, None, ws)
    assert ei.value.status == binding.NBLDPC_ERR_ARG
    # check degree 9 at q = 256 and 33 at q = 4: outside the kernels' limits
    for q, deg in ((256, 9), (4, 33)):
        rng = np.random.default_rng(q)
        n = deg + 12
        h = np.zeros((4, n), np.int64)
        h[0, :deg] = rng.integers(1, q, deg)
        for r in range(1, 4):
            h[r, deg + 4 * (r - 1): deg + 4 * r] = rng.integers(1, q, 4)
        h[1:, 0] = 1
        big = binding.Decoder.from_code(I.code_from_dense(h, q, I.PRIMITIVE_POLY[q]))
        with pytest.raises(binding.NbldpcError) as ei:
            binding.nbldpc_fftspa_workspace_size(big.handle, 4)
        assert ei.value.status == binding.NBLDPC_ERR_UNSUPPORTED


def test_full_size_sampled():
    """The GF(64) N=576 workload at full size (196,608 frames, one launch):
    sampled frames against the oracle, and the decision statistics."""
    code = I.workload_code("gf64_n576_dv2_dc4")
    w = I.WORKLOADS["gf64_n576_dv2_dc4"]
    parts, cws = [], []
    for i, eb in enumerate(w["ebn0"]):
        b = I.make_batch(code, eb, I.workload_seed("gf64_n576_dv2_dc4", i), w["frames"], device="cuda",
                         chunk=8192, prob=True)
        parts.append(b.prob)
        cws.append(b.codewords)
    prob = torch.cat(parts).contiguous()
    del parts
    dec = binding.Decoder.from_code(code)
    sym, its, ok = dec.fftspa_decode(prob, w["max_iters"], w["early_stop"])
    pick = np.random.default_rng(3).choice(prob.shape[0], 48, replace=False)
    ps = prob[torch.as_tensor(pick, device="cuda")].cpu().numpy()
    ws, wi, wo, wapp = oracle.fftspa_decode(code, ps, w["max_iters"], w["early_stop"], threads=THREADS,
                                            want_app=True)
    got = [t.cpu().numpy()[pick] for t in (sym, its, ok)]
    assert_decisions(code, got, (ws, wi, wo), wapp, "full-size sample")
    cw = torch.cat(cws)
    fer = float((sym.to(torch.int64) != cw).any(1).float().mean())
    assert fer < 0.2
    assert bool((its[ok == 0] == w["max_iters"]).all())      # early stop: unfinished frames ran I_max


@pytest.mark.parametrize("chunk", [7, 100, 4096])
def test_host_buffers_in_chunks_equal_the_device_decode(chunk):
    """nbldpc_fftspa_decode_host (pinned host rows, two streams, chunked) returns
    exactly what the device-buffer decode returns for the same frames."""
    code = I.workload_code("gf16_n1024_dv2_dc4")
    b = I.make_batch(code, 2.0, 57, 333, prob=True)
    dec = binding.Decoder.from_code(code)
    want = [t.cpu() for t in dec.fftspa_decode(b.prob.cuda(), 15, 1)]
    ph = b.prob.contiguous().pin_memory()
    sym = torch.empty((333, code.n), dtype=torch.uint8).pin_memory()
    its = torch.empty(333, dtype=torch.int32).pin_memory()
    ok = torch.empty(333, dtype=torch.uint8).pin_memory()
    ws = torch.empty(binding.nbldpc_fftspa_decode_host_workspace_size(dec.handle, chunk), dtype=torch.uint8,
                     device="cuda")
    stream = torch.cuda.Stream()
    binding.nbldpc_fftspa_decode_host(dec.handle, ph, 333, 15, 1, sym, its, ok, chunk, ws, stream=stream)
    stream.synchronize()
    for a, c in zip((sym, its, ok), want):
        assert torch.equal(a, c)
