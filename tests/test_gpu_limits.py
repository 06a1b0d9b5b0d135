"""The largest codes the decoders accept, and the first ones they refuse.

Both kernels stage the code description in shared memory, so the size limit
of a code is the block's shared memory, not the 16-bit edge indices: the
largest binary (2,4) code that fits must decode like the oracle, and a code
twice as large must be refused with NBLDPC_ERR_UNSUPPORTED (never a failed
launch)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_03567_gb300 import binding, inputs as I

pytestmark = pytest.mark.gpu
THREADS = 16


def random_gamma(code, frames, seed):
    rng = np.random.default_rng(seed)
    g = rng.integers(0, 40, (frames, code.n, code.q)).astype(np.uint8)
    hard = rng.integers(0, code.q, (frames, code.n))
    g[np.arange(frames)[:, None], np.arange(code.n)[None, :], hard] = 0
    return g


def test_largest_binary_code_decodes_and_larger_is_refused():
    created = None
    refused = []
    for n in (24000, 20000, 16000, 14000, 12000, 10000, 8000):
        code = I.make_regular_code(2, n, 2, 4, seed=n, encoder=False)
        try:
            dec = binding.Decoder.from_code(code)
        except binding.NbldpcError as e:
            assert e.status == binding.NBLDPC_ERR_UNSUPPORTED, e
            refused.append(n)
            continue
        created = (code, dec)
        break
    assert created is not None and refused, f"refused {refused}"
    code, dec = created
    g = random_gamma(code, 3, 5)
    got = [t.cpu().numpy() for t in dec.decode(torch.as_tensor(g).cuda(), 12, 1)]
    want = oracle.decode(code, g, 12, 1, threads=THREADS)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    # FFT-SPA on the same code: decisions against the float64 oracle, or a clean refusal
    p = np.exp(-g.astype(np.float64) / 8.0)
    p = (p / p.sum(-1, keepdims=True)).astype(np.float32)
    try:
        ws = binding.nbldpc_fftspa_workspace_size(dec.handle, 3)
    except binding.NbldpcError as e:
        assert e.status == binding.NBLDPC_ERR_UNSUPPORTED
        return
    assert ws > 0
    sym, its, ok = (t.cpu().numpy() for t in dec.fftspa_decode(torch.as_tensor(p).cuda(), 12, 1))
    ws_, wi, wo, wapp = oracle.fftspa_decode(code, p, 12, 1, threads=THREADS, want_app=True)
    # float32 against float64: symbols may differ only where the oracle's top two
    # a-posteriori values are within 1e-4 (a near-tie); the rest must match exactly
    top = np.sort(wapp, -1)
    near = (top[..., -1] - top[..., -2]) < 1e-4
    assert np.all((sym == ws_) | near)
    if np.array_equal(sym, ws_):
        assert np.array_equal(its, wi) and np.array_equal(ok, wo)
