"""Pins for the FFT-SPA oracle (Alg. 1, float64): each test checks it against
something other than itself -- the transform's definition, brute-force
enumeration of a check, exact marginals on a cycle-free Tanner graph, binary
belief propagation in the log-likelihood domain at q = 2, invariants.  CPU only."""
import itertools

import numpy as np
import pytest

from paper_2508_03567_gb300 import inputs as I


def clmul(a, b, q, poly):
    """Independent field multiply: shift-and-add reduced by the polynomial."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a & q:
            a ^= poly
    return r


def mul_table(q, poly):
    return np.array([[clmul(a, b, q, poly) for b in range(q)] for a in range(q)], dtype=np.int64)


def rand_prob(rng, shape):
    w = rng.random(shape) ** 3 + 1e-3
    return w / w.sum(-1, keepdims=True)


def make_code(q, checks, coef_seed):
    """Code object from a list of checks (column lists) with seeded coefficients."""
    rng = np.random.default_rng(coef_seed)
    row_ptr = np.zeros(len(checks) + 1, np.int32)
    cols, coefs = [], []
    for r, cs in enumerate(checks):
        row_ptr[r + 1] = row_ptr[r] + len(cs)
        cols += list(cs)
        coefs += list(rng.integers(1, q, len(cs)))
    n = max(max(c) for c in checks) + 1
    return I.Code(q=q, poly=I.PRIMITIVE_POLY[q], n=n, m=len(checks), row_ptr=row_ptr,
                  col_idx=np.array(cols, np.int32), coef=np.array(coefs, np.uint8))


# ------------------------------------------------------------ the transform
@pytest.mark.parametrize("q", [2, 4, 8, 16, 32, 64, 128, 256])
def test_transform_is_the_walsh_hadamard_definition(oracle_lib, q):
    """W(s) = sum_x (-1)^popcount(s & x) u(x), and applying it twice gives q u."""
    rng = np.random.default_rng(q)
    u = rng.standard_normal(q)
    s = np.arange(q)
    sign = np.array([[(-1) ** bin(a & b).count("1") for b in s] for a in s], np.float64)
    w = oracle_lib.wht(u)
    np.testing.assert_allclose(w, sign @ u, rtol=0, atol=1e-12 * q)
    np.testing.assert_allclose(oracle_lib.wht(w), q * u, rtol=0, atol=1e-11 * q)


def test_transform_turns_xor_convolution_into_a_product(oracle_lib):
    q = 16
    rng = np.random.default_rng(7)
    a, b = rng.random(q), rng.random(q)
    conv = np.array([sum(a[y] * b[x ^ y] for y in range(q)) for x in range(q)])
    np.testing.assert_allclose(oracle_lib.wht(oracle_lib.wht(a) * oracle_lib.wht(b)) / q, conv, atol=1e-12)


# ------------------------------------------------------------ the check node
def brute_force_check(q, poly, h, u):
    """v'_n(x) = sum over symbols of the other edges with
    sum_{j != n} h_j c_j = h_n x of prod_{j != n} u_j(c_j)."""
    mul = mul_table(q, poly)
    d = len(h)
    out = np.zeros((d, q))
    for n in range(d):
        others = [j for j in range(d) if j != n]
        for cs in itertools.product(range(q), repeat=d - 1):
            t = 0
            pr = 1.0
            for j, c in zip(others, cs):
                t ^= mul[h[j], c]
                pr *= u[j][c]
            # h_n x = t  ->  x = h_n^-1 t
            x = [xx for xx in range(q) if mul[h[n], xx] == t][0]
            out[n, x] += pr
    return out


@pytest.mark.parametrize("q,d", [(2, 3), (4, 3), (4, 4), (8, 3), (8, 4), (16, 3)])
def test_check_update_matches_brute_force(oracle_lib, q, d):
    """Permutation, transform, product, inverse transform and depermutation
    together give the sum-product check-node update of its definition."""
    poly = I.PRIMITIVE_POLY[q]
    rng = np.random.default_rng(100 * q + d)
    for trial in range(3):
        h = rng.integers(1, q, d).astype(np.int32)
        u = rand_prob(rng, (d, q))
        got = oracle_lib.fft_check_update(q, poly, h, u)
        np.testing.assert_allclose(got, brute_force_check(q, poly, h, u), rtol=1e-10, atol=1e-14)
        # outputs are probability vectors (the inputs sum to 1, so no normalization is needed)
        np.testing.assert_allclose(got.sum(1), 1.0, atol=1e-12)


# ---------------------------------------------- cycle-free graph: exact marginals
def brute_force_marginals(code, p):
    """APP of every symbol: sum over codewords c with c_n = x of prod_j p_j(c_j)."""
    mul = mul_table(code.q, code.poly)
    out = np.zeros((code.n, code.q))
    for word in itertools.product(range(code.q), repeat=code.n):
        ok = True
        for r in range(code.m):
            s = 0
            for e in range(code.row_ptr[r], code.row_ptr[r + 1]):
                s ^= mul[code.coef[e], word[code.col_idx[e]]]
            if s:
                ok = False
                break
        if ok:
            w = np.prod([p[i, word[i]] for i in range(code.n)])
            for i in range(code.n):
                out[i, word[i]] += w
    return out / out.sum(1, keepdims=True)


TREES = [
    (4, [[0, 1, 2], [2, 3, 4]]),
    (4, [[0, 1, 2], [2, 3, 4], [2, 5], [4, 6, 7]]),   # variable 2 on three checks
    (8, [[0, 1, 2], [2, 3, 4]]),
]


@pytest.mark.parametrize("q,checks", TREES)
def test_cycle_free_graph_gives_exact_marginals(oracle_lib, q, checks):
    """On a Tanner graph without cycles, sum-product reaches the exact symbol
    marginals once the iterations exceed the graph's depth."""
    code = make_code(q, checks, 31 * q + len(checks))
    rng = np.random.default_rng(len(checks) + q)
    for trial in range(2):
        p = rand_prob(rng, (1, code.n, q)).astype(np.float32)
        want = brute_force_marginals(code, p[0].astype(np.float64))
        sym, its, ok, app = oracle_lib.fftspa_decode(code, p, 6, 0, want_app=True)
        np.testing.assert_allclose(app[0], want, rtol=1e-9, atol=1e-12)
        assert its[0] == 6
        assert np.array_equal(sym[0], np.argmax(want, 1))


# ------------------------------------------------ q = 2: binary belief propagation
def binary_bp_llr(code, p, iters):
    """Textbook binary sum-product in the log-likelihood-ratio domain (tanh rule)."""
    n, E = code.n, code.nnz
    lch = np.log(p[:, 0].astype(np.float64)) - np.log(p[:, 1].astype(np.float64))
    cols = code.col_idx
    v2c = lch[cols].copy()
    app = lch.copy()
    for _ in range(iters):
        c2v = np.zeros(E)
        for r in range(code.m):
            es = range(code.row_ptr[r], code.row_ptr[r + 1])
            for e in es:
                t = np.prod([np.tanh(v2c[o] / 2) for o in es if o != e])
                c2v[e] = 2 * np.arctanh(np.clip(t, -1 + 1e-15, 1 - 1e-15))
        tot = lch.copy()
        np.add.at(tot, cols, c2v)
        v2c = tot[cols] - c2v
        app = tot
    return app


@pytest.mark.parametrize("dv,dc,n", [(2, 4, 24), (3, 6, 60)])
def test_q2_is_binary_belief_propagation(oracle_lib, dv, dc, n):
    code = I.make_regular_code(2, n, dv, dc, seed=dv * 100 + n)
    rng = np.random.default_rng(dv)
    llr = rng.normal(1.5, 2.0, n)                     # moderate reliabilities, some wrong signs
    p0 = 1 / (1 + np.exp(-llr))
    p = np.stack([p0, 1 - p0], 1)[None].astype(np.float32)
    for iters in (1, 3, 5):
        sym, its, ok, app = oracle_lib.fftspa_decode(code, p, iters, 0, want_app=True)
        L = binary_bp_llr(code, p[0], iters)
        np.testing.assert_allclose(app[0, :, 0], 1 / (1 + np.exp(-L)), rtol=1e-7, atol=1e-9)
        assert np.array_equal(sym[0], (L < 0).astype(np.uint8))


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("name", ["gf4_n48_dv2_dc4", "gf64_n576_dv2_dc4"])
def test_noiseless_frames_decode_at_once(oracle_lib, name):
    code = I.workload_code(name)
    b = I.make_batch(code, 3.0, 17, 3, noiseless=True, prob=True)
    sym, its, ok = oracle_lib.fftspa_decode(code, b.prob.numpy(), 10, 1)
    assert np.array_equal(sym.astype(np.int64), b.codewords.numpy())
    assert np.all(its == 0) and np.all(ok == 1)


def test_ok_flag_means_zero_syndrome_and_app_is_normalized(oracle_lib):
    code = I.workload_code("gf4_n48_dv2_dc4")
    b = I.make_batch(code, 2.0, 23, 24, prob=True)
    sym, its, ok, app = oracle_lib.fftspa_decode(code, b.prob.numpy(), 12, 1, want_app=True)
    assert np.array_equal(ok, oracle_lib.syndrome_ok(code, sym))
    np.testing.assert_allclose(app.sum(-1), 1.0, atol=1e-12)
    assert np.array_equal(sym, np.argmax(app, -1).astype(np.uint8))
    assert np.all(its[ok == 1] <= 12) and np.all(its[ok == 0] == 12)
    assert ok.mean() > 0.5


def test_edge_order_within_rows_does_not_matter(oracle_lib):
    code = I.workload_code("gf4_n48_dv2_dc4")
    rng = np.random.default_rng(3)
    ci, cf = code.col_idx.copy(), code.coef.copy()
    for r in range(code.m):
        a, z = code.row_ptr[r], code.row_ptr[r + 1]
        perm = rng.permutation(z - a) + a
        ci[a:z], cf[a:z] = code.col_idx[perm], code.coef[perm]
    shuffled = I.Code(q=code.q, poly=code.poly, n=code.n, m=code.m, row_ptr=code.row_ptr, col_idx=ci, coef=cf)
    b = I.make_batch(code, 2.0, 29, 8, prob=True)
    r1 = oracle_lib.fftspa_decode(code, b.prob.numpy(), 6, 0, want_app=True)
    r2 = oracle_lib.fftspa_decode(shuffled, b.prob.numpy(), 6, 0, want_app=True)
    np.testing.assert_allclose(r1[3], r2[3], atol=1e-12)
    assert np.array_equal(r1[0], r2[0])


def test_fftspa_corrects_more_than_it_starts_with(oracle_lib):
    """Decoding lowers the symbol error count of the channel decisions."""
    code = I.workload_code("gf16_n1024_dv2_dc4")
    b = I.make_batch(code, 2.0, 41, 6, prob=True)
    p = b.prob.numpy()
    sym, its, ok = oracle_lib.fftspa_decode(code, p, 20, 1)
    cw = b.codewords.numpy()
    assert (sym != cw).sum() < (np.argmax(p, -1) != cw).sum()


def test_normalization_fallback_gives_uniform_vectors(oracle_lib):
    """A frame whose probabilities are all zero: every normalization sum is 0, so every message
    and a-posteriori vector is the uniform 1/q (the reading for non-positive sums), and the
    decision is symbol 0 (lowest symbol on ties)."""
    code = I.workload_code("gf4_n48_dv2_dc4")
    p = np.zeros((1, code.n, code.q), np.float32)
    sym, its, ok, app = oracle_lib.fftspa_decode(code, p, 3, 0, want_app=True)
    np.testing.assert_allclose(app, 1.0 / code.q, atol=0)
    assert np.all(sym == 0) and ok[0] == 1 and its[0] == 3      # the all-zero word is a codeword


def test_channel_probabilities_match_the_reliabilities():
    """Both inputs come from the same noise: the most likely symbol of p is the symbol with
    gamma = 0 (the hard decision), p sums to 1, and p falls as gamma grows."""
    code = I.workload_code("gf16_n1024_dv2_dc4")
    b = I.make_batch(code, 2.0, 123, 4, prob=True)
    p, g = b.prob.numpy().astype(np.float64), b.gamma.numpy()
    np.testing.assert_allclose(p.sum(-1), 1.0, atol=1e-5)
    assert np.all(g[np.arange(4)[:, None], np.arange(code.n)[None, :], np.argmax(p, -1)] == 0)
    # within a symbol, a strictly larger unsaturated gamma never has a larger probability
    for f in range(2):
        for n in range(0, code.n, 97):
            order = np.argsort(g[f, n], kind="stable")
            gs, ps = g[f, n][order], p[f, n][order]
            keep = gs < 63
            assert np.all(np.diff(ps[keep])[np.diff(gs[keep]) > 0] <= 1e-7)
