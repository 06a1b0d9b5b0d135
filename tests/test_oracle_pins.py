"""Pins for the CPU oracle: each test checks it against something other than
itself (field definition, brute-force enumeration, binary min-sum, the worked
example of Eq. (1), invariants).  CPU only."""
import itertools
import os

import numpy as np
import pytest
import torch

from paper_2508_03567_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------
# An independent field multiply for the pins: shift-and-add (carry-less)
# multiplication reduced by the primitive polynomial, written out here.
# --------------------------------------------------------------------------
def clmul(a, b, q, poly):
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a & q:
            a ^= poly
    return r


def clmul_table(q, poly):
    return np.array([[clmul(a, b, q, poly) for b in range(q)] for a in range(q)], dtype=np.int64)


FIELDS = sorted(I.PRIMITIVE_POLY.items())


# ---------------------------------------------------------------- P1 field
@pytest.mark.parametrize("q,poly", FIELDS)
def test_field_matches_polynomial_arithmetic(oracle_lib, q, poly):
    """The oracle's exp/log multiply equals polynomial multiplication mod the
    primitive polynomial (Sec. 2.1: GF(2^p) built from a primitive polynomial)."""
    mul, inv = oracle_lib.gf_mul_all(q, poly)
    ref = clmul_table(q, poly)
    assert np.array_equal(mul, ref)
    a = np.arange(1, q)
    assert np.all(mul[a, inv[a]] == 1)          # inverse
    assert inv[0] == 0


@pytest.mark.parametrize("q,poly", FIELDS)
def test_field_axioms(oracle_lib, q, poly):
    mul, _ = oracle_lib.gf_mul_all(q, poly)
    x = np.arange(q)
    assert mul.min() >= 0 and mul.max() < q                    # closure
    assert np.array_equal(mul, mul.T)                           # commutativity
    assert np.array_equal(mul[1], x) and np.all(mul[0] == 0)    # identities
    # every non-zero row is a permutation of the non-zero elements (no zero divisors)
    for a in range(1, q):
        assert sorted(mul[a, 1:]) == list(range(1, q))
    rng = np.random.default_rng(q)
    n = min(q ** 3, 200000)
    a, b, c = (rng.integers(0, q, n) for _ in range(3))
    assert np.array_equal(mul[mul[a, b], c], mul[a, mul[b, c]])  # associativity
    assert np.array_equal(mul[a, b ^ c], mul[a, b] ^ mul[a, c])  # distributivity over XOR


@pytest.mark.parametrize("q,poly", FIELDS)
def test_primitive_element_order_and_barrel_shift(oracle_lib, q, poly):
    """x = 2 has order q-1; multiplying by x^k rotates the exponent-ordered
    vector by k with element 0 fixed (the barrel-shift view, Sec. 2.2)."""
    exp, log = oracle_lib.gf_tables(q, poly)
    assert sorted(exp.tolist()) == list(range(1, q))
    assert all(log[exp[i]] == i for i in range(q - 1))
    mul, _ = oracle_lib.gf_mul_all(q, poly)
    for k in range(q - 1):
        h = exp[k]
        # element at exponent position i moves to position (i + k) mod (q - 1)
        for i in range(q - 1):
            assert mul[h, exp[i]] == exp[(i + k) % (q - 1)]
        assert mul[h, 0] == 0


@pytest.mark.parametrize("q,poly", [(4, 0x5), (16, 0x1F), (8, 0x7), (8, 0x1B), (6, 0x7), (512, 0x211)])
def test_field_rejects_bad_polynomial(oracle_lib, q, poly):
    # x^2+1 reducible; x^4+x^3+x^2+x+1 irreducible but x has order 5;
    # degree-2 / degree-4 polynomials for GF(8); q not a power of two / too big
    assert oracle_lib.gf_tables(q, poly) is None


# ---------------------------------------------------------------- P2 check node
def brute_force_check(q, poly, h, alpha):
    """beta_j(a) = min over (a_i)_{i!=j} with sum_i h_i a_i = h_j a of
    max_{i!=j} alpha_i(a_i)  (the closed form the F/B recursion computes)."""
    mul = clmul_table(q, poly)
    d = len(h)
    beta = np.full((d, q), 1 << 30, dtype=np.int64)
    for j in range(d):
        others = [i for i in range(d) if i != j]
        tup = np.array(list(itertools.product(range(q), repeat=d - 1)), dtype=np.int64)
        s = np.zeros(len(tup), dtype=np.int64)
        mx = np.zeros(len(tup), dtype=np.int64)
        for col, i in enumerate(others):
            s ^= mul[h[i], tup[:, col]]
            mx = np.maximum(mx, alpha[i][tup[:, col]])
        inv_hj = [b for b in range(1, q) if mul[h[j], b] == 1][0]
        target = mul[inv_hj, s]          # the symbol a with h_j a = s
        np.minimum.at(beta[j], target, mx)
    return beta


CASES = [(q, d) for q in (2, 4, 8) for d in (2, 3, 4, 5)] + [(16, 2), (16, 3), (32, 3), (64, 3)]


@pytest.mark.parametrize("q,d", CASES)
def test_check_update_matches_brute_force(oracle_lib, q, d):
    poly = I.PRIMITIVE_POLY[q]
    rng = np.random.default_rng(1000 * q + d)
    for trial in range(6):
        h = rng.integers(1, q, d)
        if trial == 0:
            alpha = rng.integers(0, 256, (d, q))
        elif trial == 1:      # saturated extremes only
            alpha = rng.choice([0, 255], (d, q))
        elif trial == 2:      # all equal
            alpha = np.full((d, q), 17)
        elif trial == 3:      # min-normalized, small range (many ties)
            alpha = rng.integers(0, 4, (d, q))
            alpha[:, 0] = 0
        else:
            alpha = rng.integers(0, 64, (d, q))
        got = oracle_lib.check_update(q, poly, h, alpha)
        want = brute_force_check(q, poly, h.tolist(), alpha)
        assert np.array_equal(got.astype(np.int64), want), (q, d, trial)


# ---------------------------------------------------------------- P3 binary min-sum
def binary_min_sum(code, gamma, max_iters, early_stop, cap=255):
    """Textbook flooding min-sum on integer LLRs (no offset, no scaling),
    variable-to-check magnitudes capped at `cap`; L = gamma(1) - gamma(0)."""
    rp, ci = code.row_ptr, code.col_idx
    E = int(rp[-1])
    row_of = np.repeat(np.arange(code.m), np.diff(rp))
    out_sym, out_it, out_ok = [], [], []
    for g in gamma.astype(np.int64):
        lch = g[:, 1] - g[:, 0]

        def ok_of(c):
            par = np.zeros(code.m, np.int64)
            np.add.at(par, row_of, c[ci])
            return bool(np.all(par % 2 == 0))

        v2c = lch[ci].copy()
        chat = (lch < 0).astype(np.int64)
        ok = ok_of(chat)
        it = 0
        if not (early_stop and ok):
            for k in range(1, max_iters + 1):
                c2v = np.zeros(E, np.int64)
                for r in range(code.m):
                    es = np.arange(rp[r], rp[r + 1])
                    for e in es:
                        oth = es[es != e]
                        sgn = np.prod(np.where(v2c[oth] < 0, -1, 1))
                        c2v[e] = sgn * np.min(np.abs(v2c[oth]))
                tot = lch.copy()
                np.add.at(tot, ci, c2v)
                t = tot[ci] - c2v
                v2c = np.sign(t) * np.minimum(np.abs(t), cap)
                chat = (tot < 0).astype(np.int64)
                it = k
                ok = ok_of(chat)
                if early_stop and ok:
                    break
        out_sym.append(chat)
        out_it.append(it)
        out_ok.append(int(ok))
    return np.array(out_sym), np.array(out_it), np.array(out_ok)


@pytest.mark.parametrize("dv,dc,n,early", [(2, 4, 48, 1), (3, 6, 60, 0), (3, 6, 60, 1), (2, 6, 36, 1)])
def test_q2_is_binary_min_sum(oracle_lib, dv, dc, n, early):
    code = I.make_regular_code(2, n, dv, dc, seed=77 + n + dv)
    rng = np.random.default_rng(n * 10 + dv)
    f = 40
    gamma = np.zeros((f, n, 2), np.uint8)
    hard = rng.integers(0, 2, (f, n))
    mag = rng.integers(0, 40, (f, n))
    mag[: f // 2] = rng.integers(0, 256, (f // 2, n))     # large magnitudes exercise the 255 cap
    gamma[np.arange(f)[:, None], np.arange(n)[None, :], 1 - hard] = mag
    sym, its, ok = oracle_lib.decode(code, gamma, 12, early)
    ws, wi, wo = binary_min_sum(code, gamma, 12, early)
    assert np.array_equal(sym, ws)
    assert np.array_equal(its, wi)
    assert np.array_equal(ok, wo)


# ---------------------------------------------------------------- P4 syndrome
def syndrome_indep(code, words):
    mul = clmul_table(code.q, code.poly)
    s = np.zeros((words.shape[0], code.m), np.int64)
    for r in range(code.m):
        for e in range(code.row_ptr[r], code.row_ptr[r + 1]):
            s[:, r] ^= mul[code.coef[e], words[:, code.col_idx[e]].astype(np.int64)]
    return np.all(s == 0, axis=1)


@pytest.mark.parametrize("name,ebn0", [("gf4_n48_dv2_dc4", 2.0), ("gf16_n1024_dv2_dc4", 1.5)])
def test_ok_flag_means_zero_syndrome(oracle_lib, name, ebn0):
    code = I.workload_code(name)
    w = I.WORKLOADS[name]
    b = I.make_batch(code, ebn0, 99, 24 if code.n > 100 else 300)
    sym, its, ok = oracle_lib.decode(code, b.gamma.numpy(), 8, w["early_stop"], threads=8)
    ind = syndrome_indep(code, sym)
    assert np.array_equal(ok.astype(bool), ind)
    assert ok.any() and (~ok.astype(bool)).any() or name != "gf4_n48_dv2_dc4"


# ---------------------------------------------------------------- P5 noiseless
@pytest.mark.parametrize("name", ["gf4_n48_dv2_dc4", "gf16_n1024_dv2_dc4", "gf32_n600_dv3_dc6",
                                  "gf256_n128_dv2_dc8"])
def test_noiseless_frames_decode_to_the_codeword(oracle_lib, name):
    code = I.workload_code(name)
    b = I.make_batch(code, 2.5, 5, 3, noiseless=True)
    cw = b.codewords.numpy()
    sym, its, ok = oracle_lib.decode(code, b.gamma.numpy(), 4, 1)
    assert np.array_equal(sym, cw) and np.all(its == 0) and np.all(ok == 1)
    if code.q <= 32:
        sym, its, ok = oracle_lib.decode(code, b.gamma.numpy(), 2, 0)  # fixed point
        assert np.array_equal(sym, cw) and np.all(its == 2) and np.all(ok == 1)


# ---------------------------------------------------------------- P6 order invariance
def test_edge_order_within_rows_does_not_matter(oracle_lib):
    code = I.make_regular_code(8, 40, 2, 4, seed=5)
    b = I.make_batch(code, 1.0, 11, 30)
    rng = np.random.default_rng(3)
    ci, cf = code.col_idx.copy(), code.coef.copy()
    for r in range(code.m):
        lo, hi = code.row_ptr[r], code.row_ptr[r + 1]
        pm = rng.permutation(hi - lo) + lo
        ci[lo:hi], cf[lo:hi] = ci[pm], cf[pm]
    shuffled = I.Code(q=code.q, poly=code.poly, n=code.n, m=code.m, row_ptr=code.row_ptr,
                      col_idx=ci, coef=cf, rank=code.rank)
    a = oracle_lib.decode(code, b.gamma.numpy(), 10, 1)
    s = oracle_lib.decode(shuffled, b.gamma.numpy(), 10, 1)
    for x, y in zip(a, s):
        assert np.array_equal(x, y)


# ---------------------------------------------------------------- P7 worked example
def load_eq1():
    rows = []
    with open(os.path.join(HERE, "golden", "eq1_gf4_H.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line:
                rows.append(line)
    exp = [1, 2, 3]   # alpha^0, alpha^1, alpha^2 in GF(4) with x^2 + x + 1
    return np.array([[0 if t == "-" else exp[int(t)] for t in r] for r in rows])


def test_eq1_code_codewords_enumerate(oracle_lib):
    h = load_eq1()
    assert h.shape == (3, 6)
    assert all((h != 0).sum(1) == 4) and all((h != 0).sum(0) == 2)   # regular (2,4)
    code = I.code_from_dense(h, 4, 0x7)
    words = np.array(list(itertools.product(range(4), repeat=6)), dtype=np.uint8)
    ok = oracle_lib.syndrome_ok(code, words).astype(bool)
    assert np.array_equal(ok, syndrome_indep(code, words))
    assert ok.sum() == 4 ** code.k
    # the systematic encoder reaches exactly these codewords
    info = torch.tensor(list(itertools.product(range(4), repeat=code.k)))
    cw = I.encode(code, info).numpy()
    got = {tuple(r) for r in cw}
    assert got == {tuple(r) for r in words[ok].astype(np.int64)}


def test_eq1_code_decodes_a_single_symbol_error(oracle_lib):
    h = load_eq1()
    code = I.code_from_dense(h, 4, 0x7)
    cw = np.zeros(6, np.int64)
    gamma = np.full((1, 6, 4), 40, np.uint8)
    gamma[0, np.arange(6), cw] = 0
    gamma[0, 2, :] = [12, 20, 20, 0]   # symbol 2 leans to 3, weakly
    sym, its, ok = oracle_lib.decode(code, gamma, 5, 1)
    assert ok[0] == 1 and np.array_equal(sym[0], cw) and its[0] >= 1


# ---------------------------------------------------------------- P9 one iteration by hand
def load_iteration1():
    """Sections of tests/golden/eq1_gf4_iteration1.txt as integer arrays."""
    sec, cur = {}, None
    with open(os.path.join(HERE, "golden", "eq1_gf4_iteration1.txt")) as fh:
        for line in fh:
            t = line.split("#")[0].strip()
            if not t:
                continue
            if t.startswith("["):
                cur = t.strip("[]")
                sec[cur] = []
                continue
            sec[cur].append([int(v) for v in t.split(":")[-1].split()])
    return {k: np.array(v, dtype=np.int64) for k, v in sec.items()}


def test_eq1_one_iteration_worked_by_hand(oracle_lib):
    """Alg. 2 at q = 4: one check-node pass and one variable-node pass on the Eq. (1) code, every
    message compared with the values derived by hand in the golden file."""
    g = load_iteration1()
    code = I.code_from_dense(load_eq1(), 4, 0x7)
    gamma = g["gamma"].astype(np.uint8)
    assert gamma.shape == (6, 4) and g["beta"].shape == g["alpha"].shape == (code.nnz, 4)
    for r in range(code.m):             # the check-node pass alone, row by row, from alpha^(0) = gamma
        e = slice(code.row_ptr[r], code.row_ptr[r + 1])
        beta = oracle_lib.check_update(4, 0x7, code.coef[e], gamma[code.col_idx[e]])
        assert np.array_equal(beta, g["beta"][e]), r
    beta, s, alpha, sym = oracle_lib.decode_trace(code, gamma, 1)
    assert np.array_equal(beta, g["beta"])
    assert np.array_equal(s, g["S"])
    assert np.array_equal(alpha, g["alpha"])
    assert np.array_equal(sym, g["decision"][0])
    # the stop test: the channel decision fails check 0, the decision of iteration 1 is a codeword
    sym0, its0, ok0 = oracle_lib.decode(code, gamma[None], 0, 1)
    assert sym0[0].tolist() == [0, 0, 0, 1, 0, 0] and its0[0] == 0 and ok0[0] == 0
    sym1, its1, ok1 = oracle_lib.decode(code, gamma[None], 5, 1)
    assert np.array_equal(sym1[0], g["decision"][0]) and its1[0] == 1 and ok1[0] == 1


def test_eq1_worked_iteration_tells_the_planted_mistakes_apart():
    """The hand-worked case separates the readings a plausible mistake would change: for some edges
    the variable-node sum gamma + (other beta) is smallest at a non-zero symbol, so normalizing by
    its value at symbol 0 would give other messages; and column 3's a-posteriori sum ties at its
    minimum, so the highest-symbol tie-break would decide 1 there, which fails check 0."""
    g = load_iteration1()
    code = I.code_from_dense(load_eq1(), 4, 0x7)
    gamma, beta, alpha = g["gamma"], g["beta"], g["alpha"]
    shifted = 0
    for n in range(code.n):
        edges = np.nonzero(code.col_idx == n)[0]
        assert len(edges) == 2
        for e, other in ((edges[0], edges[1]), (edges[1], edges[0])):
            a_prime = gamma[n] + beta[other]
            assert np.array_equal(alpha[e], a_prime - a_prime.min())
            shifted += int(a_prime[0] != a_prime.min())
    assert shifted >= 3
    s3 = g["S"][3]
    assert (s3 == s3.min()).sum() == 2 and g["decision"][0][3] == 0
    word = g["decision"][0].copy()
    word[3] = int(np.nonzero(s3 == s3.min())[0].max())
    assert not syndrome_indep(code, word[None].astype(np.uint8))[0]


# ---------------------------------------------------------------- input generator
def test_inputs_are_codewords_and_reliabilities(oracle_lib):
    for name in ["gf4_n48_dv2_dc4", "gf64_n576_dv2_dc4", "gf32_n600_dv3_dc6"]:
        code = I.workload_code(name)
        b = I.make_batch(code, 2.0, 3, 16)
        assert oracle_lib.syndrome_ok(code, b.codewords.numpy().astype(np.uint8)).all()
        g = b.gamma.numpy()
        assert g.max() <= 63 and np.all(g.min(-1) == 0)
        # frames are independent of the batch split (block-seeded streams)
        part = I.make_batch(code, 2.0, 3, 5, frame0=9)
        assert torch.equal(part.gamma, b.gamma[9:14])


def test_code_construction_properties():
    for name, w in I.WORKLOADS.items():
        code = I.workload_code(name)
        deg_r = np.diff(code.row_ptr)
        deg_c = np.bincount(code.col_idx, minlength=code.n)
        assert np.all(deg_r == w["dc"]) and np.all(deg_c == w["dv"])
        assert code.coef.min() >= 1 and code.coef.max() < code.q
        # girth > 4: no two columns share two rows
        pairs = set()
        for r in range(code.m):
            cols = sorted(code.col_idx[code.row_ptr[r]:code.row_ptr[r + 1]])
            assert len(set(cols)) == len(cols)
            for a, b in itertools.combinations(cols, 2):
                assert (a, b) not in pairs
                pairs.add((a, b))


def test_vnp_saturates_at_255(oracle_lib):
    """A hand-worked binary case where the variable-node cap decides a symbol.

    H = [[1,1,0],[1,0,1]]; v0 leans to 0 by 255, v1 to 1 by 255, v2 to 0 by 255.
    Iteration 1: v0 receives +255 from check 1 and -255 from check 0, so its
    message to check 0 is 255 + 255 = 510, capped to 255.  Iteration 2:
    check 0 forwards that 255 to v1, whose posterior is then 255 - 255 = 0 in
    LLR, a tie, decided as the lowest symbol, 0.  A cap of 254 would give 1.
    """
    code = I.code_from_dense(np.array([[1, 1, 0], [1, 0, 1]]), 2, 0x3)
    gamma = np.array([[[0, 255], [255, 0], [0, 255]]], np.uint8)
    sym, its, ok = oracle_lib.decode(code, gamma, 2, 0)
    assert sym.tolist() == [[0, 0, 0]] and its.tolist() == [2] and ok.tolist() == [1]
    ws, wi, wo = binary_min_sum(code, gamma, 2, 0)
    assert np.array_equal(sym, ws)


# ---------------------------------------------------------------- 16-bit messages
@pytest.mark.parametrize("dv,dc,n", [(3, 6, 60), (2, 4, 48)])
def test_q2_wide_messages_are_binary_min_sum_with_the_wide_cap(oracle_lib, dv, dc, n):
    code = I.make_regular_code(2, n, dv, dc, seed=91 + n + dv)
    rng = np.random.default_rng(n + 7 * dv)
    f = 30
    gamma = np.zeros((f, n, 2), np.uint8)
    hard = rng.integers(0, 2, (f, n))
    gamma[np.arange(f)[:, None], np.arange(n)[None, :], 1 - hard] = rng.integers(100, 256, (f, n))
    for cap in (255, 65535):
        sym, its, ok = oracle_lib.decode(code, gamma, 15, 0, cap=cap)
        ws, wi, wo = binary_min_sum(code, gamma, 15, 0, cap=cap)
        assert np.array_equal(sym, ws) and np.array_equal(its, wi) and np.array_equal(ok, wo)


def test_wide_cap_never_binds_for_column_degree_two(oracle_lib):
    """With column degree 2 a message grows by at most max(gamma) per iteration
    (alpha = gamma + beta - min and beta <= the largest incoming alpha), so
    with gamma <= 63 and 30 iterations 16-bit messages equal unbounded ones."""
    code = I.workload_code("gf16_n1024_dv2_dc4")
    g = I.make_batch(code, 1.0, 31, 6).gamma.numpy()
    a = oracle_lib.decode(code, g, 30, 0, cap=65535)
    b = oracle_lib.decode(code, g, 30, 0, cap=1 << 30)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
