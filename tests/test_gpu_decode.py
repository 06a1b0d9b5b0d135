"""GPU parity: the CUDA decoder (through the C ABI) against the CPU oracle,
element by element, on seeded inputs; plus edge cases and properties that hold
at any size.  Bar: bit-exact (every output is an integer decided by integer
arithmetic with fixed tie-breaks)."""
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


def gpu_decode(code, gamma, max_iters, early_stop):
    dec = binding.Decoder.from_code(code)
    g = torch.as_tensor(gamma).cuda().contiguous()
    s, i, o = dec.decode(g, max_iters, early_stop)
    torch.cuda.synchronize()
    return s.cpu().numpy(), i.cpu().numpy(), o.cpu().numpy()


def assert_same(got, want, ctx=""):
    names = ("symbols", "iterations", "ok")
    for n, g, w in zip(names, got, want):
        if not np.array_equal(g, w):
            bad = np.nonzero((g != w).reshape(g.shape[0], -1).any(1))[0]
            raise AssertionError(f"{ctx}: {n} differ in {bad.size} frames, first {bad[:8].tolist()}")


# --------------------------------------------------------------- workloads
SMALL = [("gf4_n48_dv2_dc4", 1000), ("gf64_n576_dv2_dc4", 64), ("gf16_n1024_dv2_dc4", 48),
         ("gf32_n600_dv3_dc6", 48), ("gf256_n128_dv2_dc8", 16), ("gf256_n384_dv2_dc6", 12)]


@pytest.mark.parametrize("name,frames", SMALL)
def test_workload_parity(name, frames):
    w = I.WORKLOADS[name]
    code = I.workload_code(name)
    for k, eb in enumerate(w["ebn0"]):
        b = I.make_batch(code, eb, I.workload_seed(name, k) + 1, frames)
        g = b.gamma.numpy()
        got = gpu_decode(code, g, w["max_iters"], w["early_stop"])
        want = oracle.decode(code, g, w["max_iters"], w["early_stop"], threads=THREADS)
        assert_same(got, want, f"{name} @ {eb} dB")


# --------------------------------------------------------------- fields and shapes
@pytest.mark.parametrize("q,n,dv,dc", [(2, 60, 3, 6), (4, 40, 2, 5), (8, 64, 2, 4), (16, 96, 3, 6),
                                       (32, 64, 2, 4), (64, 48, 2, 6), (128, 96, 2, 4), (256, 32, 2, 4)])
def test_every_field_order(q, n, dv, dc):
    code = I.make_regular_code(q, n, dv, dc, seed=31 * q + n)
    for eb, early in ((1.0, 1), (2.5, 0)):
        b = I.make_batch(code, eb, 5 + q, 24)
        g = b.gamma.numpy()
        got = gpu_decode(code, g, 9, early)
        want = oracle.decode(code, g, 9, early, threads=THREADS)
        assert_same(got, want, f"q={q} early={early}")


def irregular_code(q, seed, dmax=9):
    """Rows of degree 2..dmax, columns of degree 1..4, random coefficients."""
    rng = np.random.default_rng(seed)
    n, m = 70, 30
    h = np.zeros((m, n), np.int64)
    for r in range(m):
        d = int(rng.integers(2, dmax + 1))
        cols = rng.choice(n, d, replace=False)
        h[r, cols] = rng.integers(1, q, d)
    for c in range(n):
        if not h[:, c].any():
            h[int(rng.integers(m)), c] = int(rng.integers(1, q))
    return I.code_from_dense(h, q, I.PRIMITIVE_POLY[q])


@pytest.mark.parametrize("q", [4, 16, 64, 256])
def test_irregular_code(q):
    code = irregular_code(q, q)
    rng = np.random.default_rng(q + 1)
    g = rng.integers(0, 40, (20, code.n, q)).astype(np.uint8)
    hard = rng.integers(0, q, (20, code.n))
    g[np.arange(20)[:, None], np.arange(code.n)[None, :], hard] = 0
    for early in (0, 1):
        got = gpu_decode(code, g, 7, early)
        want = oracle.decode(code, g, 7, early, threads=THREADS)
        assert_same(got, want, f"irregular q={q}")


def test_irregular_gf4_code_in_the_register_form():
    """Rows of degree 2..8: every check-node pass of a q = 4 code of check degree <= 8 runs in the
    register form (one lane per check) whatever each row's degree; the same frames through the
    all-field kernel of a mixed batch take the group form.  Both equal the oracle."""
    code = irregular_code(4, 43, dmax=8)          # row degrees 2..8
    assert np.diff(code.row_ptr).max() <= 8 and np.diff(code.row_ptr).min() == 2
    rng = np.random.default_rng(45)
    g = rng.integers(0, 40, (40, code.n, 4)).astype(np.uint8)
    g[np.arange(40)[:, None], np.arange(code.n)[None, :], rng.integers(0, 4, (40, code.n))] = 0
    dec = binding.Decoder.from_code(code)
    gd = torch.as_tensor(g).cuda()
    for v in (0, 1, 2, 3):
        dec.set_tuning(v, 1)
        for early in (0, 1):
            got = [t.cpu().numpy() for t in dec.decode(gd, 7, early)]
            assert_same(got, oracle.decode(code, g, 7, early, threads=THREADS), f"variant {v} early={early}")
    jobs, keep = _batch_jobs([(code, g, 7, 1)])
    ws = torch.empty(binding.nbldpc_decode_batch_workspace_size(jobs), dtype=torch.uint8, device="cuda")
    binding.nbldpc_decode_batch(jobs, ws)
    torch.cuda.synchronize()
    _, _, sym, its, ok = keep[0]
    assert_same([sym.cpu().numpy(), its.cpu().numpy(), ok.cpu().numpy()], oracle.decode(code, g, 7, 1), "batch")


# --------------------------------------------------------------- adversarial inputs
@pytest.mark.parametrize("kind", ["all_equal", "saturated", "random_u8", "zeros", "ties_small", "noiseless"])
def test_adversarial_inputs(kind):
    code = I.workload_code("gf64_n576_dv2_dc4")
    rng = np.random.default_rng(hash(kind) % 1000)
    f, n, q = 6, code.n, code.q
    if kind == "all_equal":
        g = np.full((f, n, q), 9, np.uint8)
    elif kind == "saturated":
        g = rng.choice(np.array([0, 255], np.uint8), (f, n, q))
    elif kind == "random_u8":
        g = rng.integers(0, 256, (f, n, q)).astype(np.uint8)
    elif kind == "zeros":
        g = np.zeros((f, n, q), np.uint8)
    elif kind == "ties_small":
        g = rng.integers(0, 2, (f, n, q)).astype(np.uint8)
    else:
        g = I.make_batch(code, 2.0, 3, f, noiseless=True).gamma.numpy()
    for mi, early in ((6, 1), (6, 0), (0, 0), (0, 1), (1, 0)):
        got = gpu_decode(code, g, mi, early)
        want = oracle.decode(code, g, mi, early, threads=THREADS)
        assert_same(got, want, f"{kind} max_iters={mi} early={early}")


def test_edge_counts():
    code = I.workload_code("gf16_n1024_dv2_dc4")
    b = I.make_batch(code, 1.5, 77, 3)
    g = b.gamma.numpy()
    # single frame
    assert_same(gpu_decode(code, g[:1], 30, 1), oracle.decode(code, g[:1], 30, 1), "one frame")
    # zero frames: nothing queued, no error
    dec = binding.Decoder.from_code(code)
    e = torch.empty((0, code.n, code.q), dtype=torch.uint8, device="cuda")
    s, i, o = dec.decode(e, 5, 1)
    torch.cuda.synchronize()
    assert s.shape == (0, code.n)


# --------------------------------------------------------------- batch independence, determinism
def test_frames_independent_of_batch_and_repeatable():
    code = I.workload_code("gf32_n600_dv3_dc6")
    b = I.make_batch(code, 2.0, 12, 600)
    dec = binding.Decoder.from_code(code)
    g = b.gamma.cuda()
    full = [t.cpu().numpy() for t in dec.decode(g, 30, 1)]
    again = [t.cpu().numpy() for t in dec.decode(g, 30, 1)]
    assert_same(again, full, "repeat")
    for lo, hi in ((0, 1), (17, 300), (599, 600), (100, 600)):
        part = [t.cpu().numpy() for t in dec.decode(g[lo:hi].contiguous(), 30, 1)]
        assert_same(part, [x[lo:hi] for x in full], f"slice {lo}:{hi}")


def test_host_buffer_entry_point_matches_device_path():
    code = I.workload_code("gf64_n576_dv2_dc4")
    b = I.make_batch(code, 1.5, 21, 700)
    dec = binding.Decoder.from_code(code)
    dev = [t.cpu().numpy() for t in dec.decode(b.gamma.cuda(), 20, 1)]
    gh = b.gamma.pin_memory()
    f = gh.shape[0]
    sym = torch.empty((f, code.n), dtype=torch.uint8).pin_memory()
    its = torch.empty((f,), dtype=torch.int32).pin_memory()
    ok = torch.empty((f,), dtype=torch.uint8).pin_memory()
    chunk = 256
    ws = torch.empty(binding.nbldpc_decode_host_workspace_size(dec.handle, chunk), dtype=torch.uint8,
                     device="cuda")
    s = torch.cuda.Stream()
    binding.nbldpc_decode_host(dec.handle, gh, f, 20, 1, sym, its, ok, chunk, ws, stream=s)
    s.synchronize()
    assert_same([sym.numpy(), its.numpy(), ok.numpy()], dev, "host path")


def test_workspace_too_small_is_rejected():
    code = I.workload_code("gf4_n48_dv2_dc4")
    dec = binding.Decoder.from_code(code)
    g = torch.zeros((4, code.n, code.q), dtype=torch.uint8, device="cuda")
    out = torch.empty((4, code.n), dtype=torch.uint8, device="cuda")
    it = torch.empty(4, dtype=torch.int32, device="cuda")
    ok = torch.empty(4, dtype=torch.uint8, device="cuda")
    need = binding.nbldpc_decode_workspace_size(dec.handle, 4)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(binding.NbldpcError) as ei:
        binding.nbldpc_decode(dec.handle, g, 4, 5, 1, out, it, ok, ws, workspace_bytes=need - 1)
    assert ei.value.status == binding.NBLDPC_ERR_ARG


# --------------------------------------------------------------- full size, as benchmarked
def test_full_size_gf64_batch_sampled_parity():
    """The benchmark's launch: 65536 frames at each of 1.5/2.0/2.5 dB in one
    call; sampled frames against the oracle, every frame against the
    syndrome property."""
    name = "gf64_n576_dv2_dc4"
    w = I.WORKLOADS[name]
    code = I.workload_code(name)
    parts = [I.make_batch(code, eb, I.workload_seed(name, k), w["frames"], device="cuda", chunk=8192).gamma
             for k, eb in enumerate(w["ebn0"])]
    g = torch.cat(parts, 0).contiguous()
    del parts
    dec = binding.Decoder.from_code(code)
    s, i, o = dec.decode(g, w["max_iters"], w["early_stop"])
    torch.cuda.synchronize()
    s, i, o = s.cpu().numpy(), i.cpu().numpy(), o.cpu().numpy()
    f = g.shape[0]
    rng = np.random.default_rng(0)
    pick = np.unique(np.concatenate([rng.choice(f, 40, replace=False), [0, f - 1, 65535, 65536, 131071]]))
    gs = g[torch.as_tensor(pick, device="cuda")].cpu().numpy()
    want = oracle.decode(code, gs, w["max_iters"], w["early_stop"], threads=THREADS)
    assert_same([s[pick], i[pick], o[pick]], want, "sampled full-size frames")
    assert i.min() >= 0 and i.max() <= w["max_iters"]
    okv = oracle.syndrome_ok(code, s)
    assert np.array_equal(okv, o)
    assert np.all(i[o == 0] == w["max_iters"])      # early stop: a failed frame ran all iterations


def test_full_size_gf256_batch_sampled_parity():
    name = "gf256_n384_dv2_dc6"
    w = I.WORKLOADS[name]
    code = I.workload_code(name)
    g = I.make_batch(code, w["ebn0"][0], I.workload_seed(name, 0), w["frames"], device="cuda",
                     chunk=2048).gamma
    dec = binding.Decoder.from_code(code)
    s, i, o = dec.decode(g, w["max_iters"], w["early_stop"])
    torch.cuda.synchronize()
    s, i, o = s.cpu().numpy(), i.cpu().numpy(), o.cpu().numpy()
    pick = np.array([0, 1, 4097, 9000, 16383])
    want = oracle.decode(code, g[torch.as_tensor(pick, device="cuda")].cpu().numpy(), w["max_iters"],
                         w["early_stop"], threads=THREADS)
    assert_same([s[pick], i[pick], o[pick]], want, "sampled GF(256) frames")
    assert np.array_equal(oracle.syndrome_ok(code, s), o)


def test_generator_is_device_independent():
    code = I.workload_code("gf64_n576_dv2_dc4")
    a = I.make_batch(code, 2.0, 99, 40, device="cpu")
    b = I.make_batch(code, 2.0, 99, 40, device="cuda")
    assert torch.equal(a.gamma, b.gamma.cpu()) and torch.equal(a.codewords, b.codewords.cpu())


# --------------------------------------------------------------- layout variants and frames per block
TUNE_CODES = [("gf4_n48_dv2_dc4", None), ("gf64_n576_dv2_dc4", None), ("gf32_n600_dv3_dc6", None),
              ("gf256_n128_dv2_dc8", None), ("q2", (2, 60, 3, 6)), ("q8", (8, 64, 2, 4)),
              ("q16", (16, 96, 2, 4)), ("q128", (128, 96, 2, 4))]


@pytest.mark.parametrize("name,shape", TUNE_CODES)
def test_every_variant_and_frames_per_block(name, shape):
    if shape is None:
        code = I.workload_code(name)
        eb = 1.5
    else:
        q, n, dv, dc = shape
        code = I.make_regular_code(q, n, dv, dc, seed=7 * q + n)
        eb = 1.0
    frames = 20
    g = I.make_batch(code, eb, 404, frames).gamma.numpy()
    want = oracle.decode(code, g, 8, 1, threads=THREADS)
    dec = binding.Decoder.from_code(code)
    gd = torch.as_tensor(g).cuda()
    tried, resident, pruned = 0, 0, 0
    # bit 1: messages resident in shared memory (q >= 16, one frame per block);
    # bit 2: pruned convolutions (layouts of 32-lane groups: GF(64) layout 0, GF(128), GF(256))
    for v in range(8):
        for fpb in (1, 2, 4, 8):
            try:
                dec.set_tuning(v, fpb)
            except binding.NbldpcError as e:
                assert e.status == binding.NBLDPC_ERR_UNSUPPORTED
                continue
            assert dec.tuning() == (v, fpb)
            got = [t.cpu().numpy() for t in dec.decode(gd, 8, 1)]
            assert_same(got, want, f"{name} variant {v} fpb {fpb}")
            tried += 1
            resident += (v & 2) != 0
            pruned += (v & 4) != 0
    assert tried >= 2
    assert resident >= 2            # both layouts with messages in shared memory, one frame per block at least
    if code.q >= 64:
        assert pruned >= 4          # every frames-per-block count of at least one pruned layout


def test_autotune_picks_a_valid_pair_and_keeps_results():
    code = I.workload_code("gf16_n1024_dv2_dc4")
    g = I.make_batch(code, 2.0, 505, 64).gamma
    dec = binding.Decoder.from_code(code)
    res = dec.autotune(g.cuda(), 3)
    assert len(res) >= 2 and all(ms > 0 for _, _, ms in res)
    best = min(res, key=lambda r: r[2])
    assert dec.tuning() == (best[0], best[1])
    got = [t.cpu().numpy() for t in dec.decode(g.cuda(), 30, 1)]
    assert_same(got, oracle.decode(code, g.numpy(), 30, 1, threads=THREADS), "after autotune")


# --------------------------------------------------------------- mixed-code batches
def _batch_jobs(specs):
    jobs, keep = [], []
    for code, g, mi, es in specs:
        dec = binding.Decoder.from_code(code)
        f = g.shape[0]
        gd = torch.as_tensor(g).cuda().contiguous()
        sym = torch.empty((f, code.n), dtype=torch.uint8, device="cuda")
        its = torch.empty((f,), dtype=torch.int32, device="cuda")
        ok = torch.empty((f,), dtype=torch.uint8, device="cuda")
        keep.append((dec, gd, sym, its, ok))
        jobs.append((dec.handle, gd, f, mi, es, sym, its, ok))
    return jobs, keep


def test_mixed_code_batch_matches_oracle():
    specs = []
    for name, frames, eb in (("gf16_n1024_dv2_dc4", 37, 1.5), ("gf64_n576_dv2_dc4", 5, 2.0),
                             ("gf32_n600_dv3_dc6", 23, 2.5), ("gf256_n128_dv2_dc8", 11, 3.5),
                             ("gf4_n48_dv2_dc4", 300, 3.0), ("gf256_n384_dv2_dc6", 0, 2.5)):
        w = I.WORKLOADS[name]
        code = I.workload_code(name)
        g = I.make_batch(code, eb, 606, frames).gamma.numpy() if frames else \
            np.zeros((0, code.n, code.q), np.uint8)
        specs.append((code, g, w["max_iters"], w["early_stop"]))
    jobs, keep = _batch_jobs(specs)
    ws = torch.empty(binding.nbldpc_decode_batch_workspace_size(jobs), dtype=torch.uint8, device="cuda")
    before = binding.nbldpc_kernel_launch_count()
    binding.nbldpc_decode_batch(jobs, ws)
    torch.cuda.synchronize()
    assert binding.nbldpc_kernel_launch_count() == before + 1
    for (code, g, mi, es), (_, _, sym, its, ok) in zip(specs, keep):
        if g.shape[0] == 0:
            continue
        want = oracle.decode(code, g, mi, es, threads=THREADS)
        assert_same([sym.cpu().numpy(), its.cpu().numpy(), ok.cpu().numpy()], want, f"batch q={code.q}")


def test_mixed_batch_replays_from_a_cuda_graph():
    names = ("gf16_n1024_dv2_dc4", "gf256_n128_dv2_dc8")
    specs = []
    for name in names:
        w = I.WORKLOADS[name]
        code = I.workload_code(name)
        specs.append((code, I.make_batch(code, 2.0, 707, 16).gamma.numpy(), w["max_iters"], w["early_stop"]))
    jobs, keep = _batch_jobs(specs)
    ws = torch.empty(binding.nbldpc_decode_batch_workspace_size(jobs), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    binding.nbldpc_decode_batch(jobs, ws, stream=s)      # first call outside capture
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        binding.nbldpc_decode_batch(jobs, ws, stream=s)
    for rnd in range(2):
        # new inputs in the same buffers, then replay
        for (code, _, mi, es), (dec, gd, sym, its, ok) in zip(specs, keep):
            fresh = I.make_batch(code, 1.5 + rnd, 808 + rnd, 16).gamma
            gd.copy_(fresh.cuda())
        graph.replay()
        torch.cuda.synchronize()
        for (code, _, mi, es), (dec, gd, sym, its, ok) in zip(specs, keep):
            want = oracle.decode(code, gd.cpu().numpy(), mi, es, threads=THREADS)
            assert_same([sym.cpu().numpy(), its.cpu().numpy(), ok.cpu().numpy()], want, f"replay {rnd}")


# --------------------------------------------------------------- 16-bit messages
WIDE = [("gf64_n576_dv2_dc4", None, 24, 1.5), ("gf32_n600_dv3_dc6", None, 24, 1.0),
        ("gf256_n128_dv2_dc8", None, 8, 2.0), ("q2", (2, 60, 3, 6), 30, 0.0), ("q8", (8, 64, 3, 6), 24, 0.5),
        ("q128", (128, 96, 2, 4), 12, 1.5)]


@pytest.mark.parametrize("name,shape,frames,eb", WIDE)
def test_sixteen_bit_messages_match_the_oracle_with_the_wide_cap(name, shape, frames, eb):
    if shape is None:
        code = I.workload_code(name)
    else:
        q, n, dv, dc = shape
        code = I.make_regular_code(q, n, dv, dc, seed=13 * q + n)
    g = I.make_batch(code, eb, 4040, frames).gamma.numpy()
    if code.q == 2:   # large magnitudes: with column degree 3 the messages reach the 65535 cap
        g = (g.astype(np.int32) * 4).clip(0, 255).astype(np.uint8)
    dec = binding.Decoder.from_code(code)
    dec.set_message_bits(16)
    assert dec.message_bits() == 16
    gd = torch.as_tensor(g).cuda()
    for mi, early in ((25, 1), (12, 0)):
        got = [t.cpu().numpy() for t in dec.decode(gd, mi, early)]
        want = oracle.decode(code, g, mi, early, threads=THREADS, cap=65535)
        assert_same(got, want, f"{name} 16-bit max_iters={mi} early={early}")
    for v in (0, 1):
        for fpb in (1, 2):
            try:
                dec.set_tuning(v, fpb)
            except binding.NbldpcError:
                continue
            got = [t.cpu().numpy() for t in dec.decode(gd, 25, 1)]
            assert_same(got, oracle.decode(code, g, 25, 1, threads=THREADS, cap=65535), f"{name} v{v} fpb{fpb}")
    dec.set_message_bits(8)
    got = [t.cpu().numpy() for t in dec.decode(gd, 25, 1)]
    assert_same(got, oracle.decode(code, g, 25, 1, threads=THREADS), f"{name} back to 8-bit")


def test_mixed_batch_rejects_sixteen_bit_codes():
    code = I.workload_code("gf16_n1024_dv2_dc4")
    dec = binding.Decoder.from_code(code)
    dec.set_message_bits(16)
    g = torch.zeros((2, code.n, code.q), dtype=torch.uint8, device="cuda")
    out = (torch.empty((2, code.n), dtype=torch.uint8, device="cuda"), torch.empty(2, dtype=torch.int32, device="cuda"),
           torch.empty(2, dtype=torch.uint8, device="cuda"))
    with pytest.raises(binding.NbldpcError) as ei:
        binding.nbldpc_decode_batch_workspace_size([(dec.handle, g, 2, 5, 1, *out)])
    assert ei.value.status == binding.NBLDPC_ERR_UNSUPPORTED


# --------------------------------------------------------------- Table 1 check-node schedule
@pytest.mark.parametrize("name", ["gf64_n576_dv2_dc4", "gf32_n600_dv3_dc6", "gf256_n128_dv2_dc8", "gf4_n48_dv2_dc4"])
def test_table1_schedule_gives_identical_outputs(name):
    """3 d_c - 4 convolutions per check (F_{d-1}, B_0 computed and unused): same results as the oracle,
    for both layout variants."""
    code = I.workload_code(name)
    g = I.make_batch(code, 1.5, 8080, 16).gamma.numpy()
    dec = binding.Decoder.from_code(code)
    binding.nbldpc_code_set_cnp_schedule(dec.handle, binding.NBLDPC_CNP_TABLE1)
    assert binding.nbldpc_code_get_cnp_schedule(dec.handle) == binding.NBLDPC_CNP_TABLE1
    gd = torch.as_tensor(g).cuda()
    want = oracle.decode(code, g, 20, 1, threads=THREADS)
    for v in (0, 1):
        dec.set_tuning(v, 1)
        assert_same([t.cpu().numpy() for t in dec.decode(gd, 20, 1)], want, f"{name} table1 v{v}")
    binding.nbldpc_code_set_cnp_schedule(dec.handle, binding.NBLDPC_CNP_MINIMAL)
    assert_same([t.cpu().numpy() for t in dec.decode(gd, 20, 1)], want, f"{name} back to minimal")


def test_table1_schedule_limits():
    """The Table 1 schedule is an 8-bit single-code kernel: 16-bit messages and mixed batches refuse it."""
    code = I.workload_code("gf16_n1024_dv2_dc4")
    dec = binding.Decoder.from_code(code)
    binding.nbldpc_code_set_cnp_schedule(dec.handle, binding.NBLDPC_CNP_TABLE1)
    with pytest.raises(binding.NbldpcError) as ei:
        dec.set_message_bits(16)
    assert ei.value.status == binding.NBLDPC_ERR_UNSUPPORTED
    g = torch.zeros((2, code.n, code.q), dtype=torch.uint8, device="cuda")
    out = (torch.empty((2, code.n), dtype=torch.uint8, device="cuda"), torch.empty(2, dtype=torch.int32, device="cuda"),
           torch.empty(2, dtype=torch.uint8, device="cuda"))
    with pytest.raises(binding.NbldpcError) as ei:
        binding.nbldpc_decode_batch_workspace_size([(dec.handle, g, 2, 5, 1, *out)])
    assert ei.value.status == binding.NBLDPC_ERR_UNSUPPORTED
    binding.nbldpc_code_set_cnp_schedule(dec.handle, binding.NBLDPC_CNP_MINIMAL)
    dec.set_message_bits(16)
    with pytest.raises(binding.NbldpcError) as ei:
        binding.nbldpc_code_set_cnp_schedule(dec.handle, binding.NBLDPC_CNP_TABLE1)
    assert ei.value.status == binding.NBLDPC_ERR_UNSUPPORTED


# --------------------------------------------------------------- the hand-worked GF(4) iteration
def test_eq1_worked_iteration_on_the_gpu():
    """The Eq. (1) code and channel values of tests/golden/eq1_gf4_iteration1.txt: the decision after
    1..3 iterations (every layout variant and frames-per-block count) equals the oracle's, and the
    hand-derived decision of iteration 1 with the stop test after it."""
    from test_oracle_pins import load_eq1, load_iteration1
    g = load_iteration1()
    code = I.code_from_dense(load_eq1(), 4, 0x7)
    gamma = np.repeat(g["gamma"].astype(np.uint8)[None], 40, 0)
    dec = binding.Decoder.from_code(code)
    gt = torch.as_tensor(gamma).cuda()
    for v in (0, 1):
        for fpb in (1, 2, 4, 8):
            dec.set_tuning(v, fpb)
            for iters in (1, 2, 3):
                got = [t.cpu().numpy() for t in dec.decode(gt, iters, 0)]
                assert_same(got, oracle.decode(code, gamma, iters, 0), f"v{v} fpb{fpb} {iters} it")
            s, i, o = (t.cpu().numpy() for t in dec.decode(gt, 5, 1))
            assert np.all(s == g["decision"][0]) and np.all(i == 1) and np.all(o == 1)


# --------------------------------------------------------------- GF(4): one warp per frame
def small_gf4_code(seed, m=20, n=36, max_row=4, max_col=2):
    """Rows of degree 2..max_row, columns of degree 1..max_col, at least one column of degree 1 and
    one of degree max_col: column sockets dealt to rows of drawn degrees (no repeated column)."""
    rng = np.random.default_rng(seed)
    for _ in range(10000):
        col_deg = rng.integers(1, max_col + 1, n)
        col_deg[0], col_deg[1] = 1, max_col
        e = int(col_deg.sum())
        if not 2 * m <= e <= max_row * m:
            continue
        row_deg = np.full(m, 2)
        for r in rng.permutation(np.repeat(np.arange(m), max_row - 2))[: e - 2 * m]:
            row_deg[r] += 1
        sockets = rng.permutation(np.repeat(np.arange(n), col_deg))
        rows = np.repeat(np.arange(m), row_deg)
        h = np.zeros((m, n), np.int64)
        if len(set(zip(rows.tolist(), sockets.tolist()))) < e:
            continue
        h[rows, sockets] = rng.integers(1, 4, e)
        return I.code_from_dense(h, 4, I.PRIMITIVE_POLY[4])
    raise RuntimeError("no code")


@pytest.mark.parametrize("shape", ["workload", "degree1_columns", "degree3_columns", "m40"])
def test_gf4_one_warp_per_frame(shape):
    """Variants 2 and 3 at 8 frames per block give each GF(4) frame one warp: codes of <= 32 checks
    of degree <= 4 and columns of degree <= 2 take the one-warp form, others the group or register
    form in the same 32-thread slot; every output equals the oracle's, with and without early stop,
    on channel frames and on the adversarial inputs."""
    if shape == "workload":
        code = I.workload_code("gf4_n48_dv2_dc4")
    elif shape == "degree1_columns":
        code = small_gf4_code(5)
        assert np.bincount(code.col_idx, minlength=code.n).min() == 1
    elif shape == "degree3_columns":
        code = small_gf4_code(6, max_col=3)
    else:
        code = small_gf4_code(7, m=40, n=72)
    rng = np.random.default_rng(11)
    f, n = 24, code.n
    gs = [I.make_batch(code, eb, 31 + k, f).gamma.numpy() for k, eb in enumerate((1.0, 3.0))]
    gs += [np.full((6, n, 4), 9, np.uint8), rng.choice(np.array([0, 255], np.uint8), (6, n, 4)),
           rng.integers(0, 256, (6, n, 4)).astype(np.uint8), np.zeros((6, n, 4), np.uint8)]
    dec = binding.Decoder.from_code(code)
    for v in (2, 3):
        dec.set_tuning(v, 8)
        assert dec.tuning() == (v, 8)
        for g in gs:
            gd = torch.as_tensor(g).cuda()
            for mi, early in ((10, 0), (10, 1), (0, 1), (1, 0)):
                got = [t.cpu().numpy() for t in dec.decode(gd, mi, early)]
                assert_same(got, oracle.decode(code, g, mi, early, threads=THREADS),
                            f"{shape} variant {v} max_iters={mi} early={early}")
