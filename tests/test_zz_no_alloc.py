"""The non-allocating decode entry point (nbldpc_decode_noalloc) against the
ordinary one.

Some callers cannot allocate device memory or hand the library a workspace
(for example a receiver that must not allocate once it runs, or code inside a
framework whose allocator owns all device memory).  For them the library
decodes in a fixed device array of its own.  This test calls that entry point
through the C ABI twice in a row and requires the same symbols, iteration
counts and ok flags as nbldpc_decode, bit for bit (the tolerance of every
decoder test here).  It lives in its own file, collected last, so that a run
stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest
import torch

from paper_2508_03567_gb300 import binding, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name,frames,ebn0", [("gf64_n576_dv2_dc4", 700, 1.5),
                                              ("gf256_n384_dv2_dc6", 400, 2.5),
                                              ("gf4_n48_dv2_dc4", 1000, 3.0)])
def test_noalloc_matches_workspace_entry_point_twice(name, frames, ebn0):
    w = I.WORKLOADS[name]
    code = I.workload_code(name)
    g = I.make_batch(code, ebn0, 606, frames, device="cuda").gamma
    dec = binding.Decoder.from_code(code)
    want = [t.cpu().numpy() for t in dec.decode(g, w["max_iters"], w["early_stop"])]
    for call in range(2):
        sym = torch.full((frames, code.n), 0xAB, dtype=torch.uint8, device="cuda")
        its = torch.full((frames,), -1, dtype=torch.int32, device="cuda")
        ok = torch.full((frames,), 7, dtype=torch.uint8, device="cuda")
        binding.nbldpc_decode_noalloc(dec.handle, g, frames, w["max_iters"], w["early_stop"], sym, its, ok)
        torch.cuda.synchronize()
        got = [sym.cpu().numpy(), its.cpu().numpy(), ok.cpu().numpy()]
        for n, a, b in zip(("symbols", "iterations", "ok"), got, want):
            assert np.array_equal(a, b), f"{name}: call {call}: {n} differ"
