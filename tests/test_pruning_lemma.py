"""The pruning lemma behind the pruned check-node convolution, checked on the CPU.

For C(x) = min_y max(A(y), B(x ^ y)) and any T >= max_x C(x), every y with
A(y) > T gives max(A(y), B(x ^ y)) > T >= C(x), so C(x) is the minimum over the
y with A(y) <= T alone (and likewise over the z with B(z) <= T, C being
symmetric in A and B).  The decoder finds such a T in phases: fold in the
entries <= hi, take M = max_x of the partial minimum (never below max_x C(x)),
stop when M <= hi, else raise hi towards M.  These tests restate that phase
algorithm in numpy and compare it with the brute-force convolution on vectors
of every shape the decoder meets (and some it should not), so a wrong bound or
a dropped entry fails here before any kernel runs."""
import numpy as np
import pytest


def dense(a, b):
    q = a.size
    x = np.arange(q)
    return np.array([np.maximum(a, b[xx ^ x]).min() for xx in range(q)])


def pruned(a, b, tprev, back=4, max_phases=6):
    """(C, entries folded, phases) by the phase algorithm."""
    q = a.size
    ca, cb = int((a <= tprev).sum()), int((b <= tprev).sum())
    u, v = (b, a) if cb < ca else (a, b)
    left = np.ones(q, bool)
    c = np.full(q, 0xFFFF, np.int64)
    hi, folded, x = max(tprev - back, 0), 0, np.arange(q)
    for phase in range(1, 64):
        sel = left & (u <= hi)
        for y in np.nonzero(sel)[0]:
            c = np.minimum(c, np.maximum(u[y], v[x ^ y]))
        folded += int(sel.sum())
        left &= ~sel
        m = int(c.max())
        if m <= hi or hi >= 0xFFFF:
            return c, folded, phase
        if m == 0xFFFF:
            hi = 2 * hi + 8
        elif phase >= max_phases:
            hi = m
        else:
            hi = min(m, max(hi + 2, (hi + m + 1) // 2))
    raise AssertionError("phases did not end")


def shapes(rng, q):
    yield rng.integers(0, 256, q), rng.integers(0, 256, q)                       # uniform 8-bit
    a = np.minimum(rng.exponential(20, q), 255).astype(np.int64); a -= a.min()    # LLR-like, min 0
    b = np.minimum(rng.exponential(12, q), 255).astype(np.int64); b -= b.min()
    yield a, b
    yield np.full(q, 9), np.full(q, 9)                                            # constant
    yield np.zeros(q, np.int64), rng.integers(0, 256, q)                          # one side all zero
    s = rng.choice([0, 255], q); s[rng.integers(q)] = 0
    yield s, rng.choice([0, 255], q)                                              # two levels
    t = np.full(q, 250); t[rng.integers(q)] = 0
    yield t, np.full(q, 240)                                                      # one small entry


@pytest.mark.parametrize("q", [4, 16, 64, 256])
def test_phase_algorithm_equals_the_dense_convolution(q):
    rng = np.random.default_rng(q)
    for trial in range(6 if q == 256 else 20):
        for a, b in shapes(rng, q):
            want = dense(a, b)
            for tprev in (0, 4, 28, 255):
                got, folded, phases = pruned(a, b, tprev)
                assert np.array_equal(got, want), (q, trial, tprev)
                assert 0 < folded <= q and phases <= 16


@pytest.mark.parametrize("q", [16, 64, 256])
def test_entries_above_the_maximum_never_decide(q):
    """The lemma itself: dropping every y with A(y) > max_x C(x) (or every z with B(z) > it)
    leaves C unchanged, while dropping one y with A(y) <= max_x C(x) that decides some C(x) changes
    it (so the bound cannot be lowered in general)."""
    rng = np.random.default_rng(7 * q)
    x = np.arange(q)
    for _ in range(10):
        a = np.minimum(rng.exponential(25, q), 255).astype(np.int64)
        b = np.minimum(rng.exponential(25, q), 255).astype(np.int64)
        c = dense(a, b)
        t = c.max()
        keep = np.nonzero(a <= t)[0]
        c_a = np.array([np.maximum(a[keep], b[xx ^ keep]).min() for xx in range(q)])
        keep_b = np.nonzero(b <= t)[0]
        c_b = np.array([np.maximum(a[xx ^ keep_b], b[keep_b]).min() for xx in range(q)])
        assert np.array_equal(c_a, c) and np.array_equal(c_b, c)
        # a y whose removal raises some C(x): the unique minimiser of some x
        for xx in range(q):
            vals = np.maximum(a, b[xx ^ x])
            if (vals == vals.min()).sum() == 1:
                y = int(vals.argmin())
                assert a[y] <= t
                rest = np.delete(np.arange(q), y)
                assert np.maximum(a[rest], b[xx ^ rest]).min() > c[xx]
                break
