"""The compile-time schedule of the select-free FFT-SPA butterflies (make_fft_signs in
csrc/fftspa_kernels.cuh), checked on the CPU: the tables are printed by a host program
built from the kernel header, and a statement-by-statement model of the kernel's
distributed check-node pass (relabelled gathers, one FMA per butterfly output with the
tabled per-lane coefficients, product over the other edges with padding for absent
edges, inverse transform, tabled output signs in the 1/q scale, natural-order scatter)
must reproduce the check-node update of Alg. 1 computed by brute force: the sum over all
assignments of the other edges' symbols whose weighted sum matches, of the product of
their probabilities.  Field arithmetic and the brute force are written here."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
POLY = {8: 0b1011, 16: 0b10011, 32: 0b100101, 64: 0b1000011, 128: 0b10000011, 256: 0b100011101}
LANE_ELEMS = {8: 4, 16: 4, 32: 4, 64: 4, 128: 4, 256: 8}     # elements per lane of the kernels


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("signs") / "fft_signs_dump")
    subprocess.check_call([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2508_03567_gb300", "csrc"),
                           os.path.join(HERE, "c", "fft_signs_dump.cu"), "-o", exe])
    tabs = {}
    for line in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines():
        t = line.split()
        q, r = int(t[1]), int(t[3])
        assert r == LANE_ELEMS[q]
        i_f, i_i, i_o = t.index("fwd"), t.index("inv"), t.index("out")
        tabs[q] = dict(ok=int(t[5]), fwd=[int(x, 16) for x in t[i_f + 1:i_i]],
                       inv=[int(x, 16) for x in t[i_i + 1:i_o]], out=[int(x, 16) for x in t[i_o + 1:]])
    return tabs


def field(q):
    """Multiplication and inverse by carry-less products reduced by the polynomial."""
    def mul(a, b):
        r = 0
        while b:
            if b & 1:
                r ^= a
            b >>= 1
            a <<= 1
            if a & q:
                a ^= POLY[q]
        return r
    inv = {a: next(b for b in range(1, q) if mul(a, b) == 1) for a in range(1, q)}
    return mul, inv


def coef(mask, gl):
    return -1.0 if (mask >> gl) & 1 else 1.0


def wht_sf(V, q, masks):
    """The kernel's select-free stages: RB register stages, then the lane stages."""
    R = LANE_ELEMS[q]
    RB = R.bit_length() - 1
    G, K = q // R, q.bit_length() - 1 - RB
    inv_order = masks is not None and masks[1]
    masks = masks[0]
    V = V.copy()
    for b in range(RB):
        h = 1 << b
        for gl in range(G):
            x = coef(masks[b], gl)
            for r in range(R):
                if not r & h:
                    keep, recv = V[gl, r], V[gl, r | h]
                    V[gl, r], V[gl, r | h] = x * keep + recv, -x * keep + recv
    for s in range(K):
        k = K - 1 - s if inv_order else s
        c = 1 << (k % RB)
        old = V.copy()                      # a shuffle reads the partner's register before the stage
        for gl in range(G):
            x = coef(masks[RB + s], gl)
            for r in range(R):
                if not r & c:
                    keep, recv = old[gl, r], old[gl ^ (1 << k), r | c]
                    V[gl, r], V[gl, r | c] = x * keep + recv, -x * keep + recv
    return V


def kernel_model(q, DC, us, hs, T):
    mul, inv = field(q)
    R = LANE_ELEMS[q]
    RB = R.bit_length() - 1
    G, K = q // R, q.bit_length() - 1 - RB
    d = len(us)
    y0 = np.arange(G) * R
    y0s = y0 ^ (np.arange(G) & ((1 << min(K, RB)) - 1))     # relabelled gather base
    pad = np.ones((G, R))
    if d < DC and (DC - d) % 2:
        pad = np.zeros((G, R))
        pad[y0s == 0, 0] = 1.0
        pad = wht_sf(pad, q, (T["fwd"], False))
    W = np.ones((DC, G, R))
    for j in range(DC):
        if j < d:
            hi = inv[hs[j]]
            V = np.array([[us[j][mul(hi, int(y0s[gl]) ^ i)] for i in range(R)] for gl in range(G)])
            W[j] = wht_sf(V, q, (T["fwd"], False))
        elif j == d:
            W[j] = pad
    outs = []
    for j in range(d):
        t = np.ones((G, R))
        for k in range(DC):
            if k != j:
                t = t * W[k]
        v = wht_sf(t, q, (T["inv"], True))
        hi = inv[hs[j]]
        dst = np.zeros(q)
        for gl in range(G):
            for i in range(R):
                dst[mul(hi, int(y0[gl]) ^ i)] = max(v[gl, i] * coef(T["out"][i], gl) / q, 0.0)
        outs.append(dst)
    return outs


def brute_force(q, us, hs):
    """v_j(x) = sum over symbols c_k of the other edges with sum_k h_k c_k = h_j x of prod_k u_k(c_k)."""
    mul, _ = field(q)
    d = len(us)
    outs = []
    for j in range(d):
        acc = np.zeros(q)
        acc[0] = 1.0                        # distribution of the weighted sum of the edges seen so far
        for k in range(d):
            if k == j:
                continue
            nxt = np.zeros(q)
            for c in range(q):              # every running sum s moves to s + h_k c
                nxt[np.arange(q) ^ mul(hs[k], c)] += acc * us[k][c]
            acc = nxt
        outs.append(np.array([acc[mul(hs[j], x)] for x in range(q)]))
    return outs


def test_tables_are_consistent(tables):
    assert sorted(tables) == [8, 16, 32, 64, 128, 256]
    for q, T in tables.items():
        assert T["ok"] == 1, q
        assert len(T["fwd"]) == len(T["inv"]) == q.bit_length() - 1
        G = q // LANE_ELEMS[q]
        assert all(m < (1 << G) for m in T["fwd"] + T["inv"] + T["out"]), q


@pytest.mark.parametrize("q", [8, 16, 32, 64, 128, 256])
@pytest.mark.parametrize("DC,degrees", [(4, (2, 3, 4)), (8, (2, 5, 6, 8))])
def test_model_matches_brute_force(tables, q, DC, degrees):
    rng = np.random.default_rng(q * 10 + DC)
    for d in degrees:
        us = [rng.random(q) for _ in range(d)]
        us = [u / u.sum() for u in us]
        hs = [int(rng.integers(1, q)) for _ in range(d)]
        got = kernel_model(q, DC, us, hs, tables[q])
        want = brute_force(q, us, hs)
        for g_, w_ in zip(got, want):
            np.testing.assert_allclose(g_, w_, rtol=0, atol=1e-13)


def test_a_wrong_coefficient_is_caught(tables):
    """Flipping one lane's coefficient in one stage breaks the check update."""
    q, DC = 16, 4
    T = {k: (list(v) if isinstance(v, list) else v) for k, v in tables[q].items()}
    T["fwd"][2] ^= 1 << 1
    rng = np.random.default_rng(3)
    us = [rng.random(q) for _ in range(4)]
    hs = [3, 5, 7, 9]
    got = kernel_model(q, DC, us, hs, T)
    want = brute_force(q, us, hs)
    assert max(np.abs(g_ - w_).max() for g_, w_ in zip(got, want)) > 1e-3


# ---- the select-based form the select-free one replaced, in float32 -------------------------
def _f32(x):
    return np.float32(x)


def wht_select_based(V, q, inverse):
    """Register butterflies (a + b, a - b), then half exchanges with selects: the lower lane of a
    pair keeps register r and sends r | c, the upper lane the reverse, and the upper lane negates
    its differences; forward lane stages 0..K-1, inverse K-1..0."""
    R = LANE_ELEMS[q]
    RB = R.bit_length() - 1
    G, K = q // R, q.bit_length() - 1 - RB
    V = V.astype(np.float32).copy()
    for b in range(RB):
        h = 1 << b
        for gl in range(G):
            for r in range(R):
                if not r & h:
                    a, c_ = V[gl, r], V[gl, r | h]
                    V[gl, r], V[gl, r | h] = _f32(a + c_), _f32(a - c_)
    for s in range(K):
        k = K - 1 - s if inverse else s
        c = 1 << (k % RB)
        old = V.copy()
        for gl in range(G):
            up = (gl >> k) & 1
            p = gl ^ (1 << k)
            for r in range(R):
                if r & c:
                    continue
                keep = old[gl, r | c] if up else old[gl, r]
                recv = old[p, r | c] if up else old[p, r]     # what the partner sends
                V[gl, r] = _f32(keep + recv)
                V[gl, r | c] = _f32((-1.0 if up else 1.0) * _f32(keep - recv))
    return V


def wht_sf32(V, q, masks, inverse):
    """The select-free stages in float32: out = recv +- x * keep with one rounding (x = +-1)."""
    R = LANE_ELEMS[q]
    RB = R.bit_length() - 1
    G, K = q // R, q.bit_length() - 1 - RB
    V = V.astype(np.float32).copy()
    for b in range(RB):
        h = 1 << b
        for gl in range(G):
            x = coef(masks[b], gl)
            for r in range(R):
                if not r & h:
                    keep, recv = V[gl, r], V[gl, r | h]
                    V[gl, r], V[gl, r | h] = _f32(recv + x * keep), _f32(recv - x * keep)
    for s in range(K):
        k = K - 1 - s if inverse else s
        c = 1 << (k % RB)
        old = V.copy()
        for gl in range(G):
            x = coef(masks[RB + s], gl)
            for r in range(R):
                if not r & c:
                    keep, recv = old[gl, r], old[gl ^ (1 << k), r | c]
                    V[gl, r], V[gl, r | c] = _f32(recv + x * keep), _f32(recv - x * keep)
    return V


def check_node_f32(q, DC, us, hs, T):
    """One check in float32 through both forms; returns (select-based, select-free) outputs."""
    mul, inv = field(q)
    R = LANE_ELEMS[q]
    RB = R.bit_length() - 1
    G, K = q // R, q.bit_length() - 1 - RB
    d = len(us)
    y0 = np.arange(G) * R
    y0s = y0 ^ (np.arange(G) & ((1 << min(K, RB)) - 1))
    outs = []
    for select_free in (False, True):
        base = y0s if select_free else y0
        W = np.ones((DC, G, R), np.float32)
        pad = np.ones((G, R), np.float32)
        if select_free and d < DC and (DC - d) % 2:
            pad = np.zeros((G, R), np.float32)
            pad[y0s == 0, 0] = 1.0
            pad = wht_sf32(pad, q, T["fwd"], False)
        for j in range(d):
            hi = inv[hs[j]]
            V = np.array([[us[j][mul(hi, int(base[gl]) ^ i)] for i in range(R)] for gl in range(G)], np.float32)
            W[j] = wht_sf32(V, q, T["fwd"], False) if select_free else wht_select_based(V, q, False)
        if d < DC:
            W[d] = pad
        res = []
        for j in range(d):
            t = np.ones((G, R), np.float32)
            for k in range(DC):                 # the kernel's product order: k = 0..DC-1, skipping j
                if k != j:
                    t = (t * W[k]).astype(np.float32)
            v = wht_sf32(t, q, T["inv"], True) if select_free else wht_select_based(t, q, True)
            hi = inv[hs[j]]
            dst = np.zeros(q, np.float32)
            for gl in range(G):
                for i in range(R):
                    tt = _f32(v[gl, i] * coef(T["out"][i], gl)) if select_free else v[gl, i]
                    dst[mul(hi, int(y0[gl]) ^ i)] = max(_f32(tt * np.float32(1.0 / q)), np.float32(0.0))
            res.append(dst)
        outs.append(res)
    return outs


@pytest.mark.parametrize("q", [8, 16, 32, 64, 128, 256])
def test_select_free_outputs_are_bit_identical_in_float32(tables, q):
    """Each select-free butterfly output is +- the select-based one with the same single rounding,
    so after the signs are folded back the check-node outputs agree bit for bit."""
    rng = np.random.default_rng(q + 7)
    for DC, d in ((4, 4), (4, 3), (8, 5), (8, 8)):
        us = [rng.random(q).astype(np.float32) for _ in range(d)]
        us = [(u / u.sum()).astype(np.float32) for u in us]
        hs = [int(rng.integers(1, q)) for _ in range(d)]
        old, new = check_node_f32(q, DC, us, hs, tables[q])
        for a, b in zip(old, new):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), (q, DC, d)
