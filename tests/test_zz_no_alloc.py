"""The non-allocating decode entry point (nbldpc_decode_noalloc) against the
ordinary one.

Some callers cannot allocate device memory or hand the library a workspace
(for example a receiver that must not allocate once it runs, or code inside a
framework whose allocator owns all device memory).  For them the library
decodes in a fixed device array of its own.  This test calls that entry point
through the C ABI twice in a row and requires the same symbols, iteration
counts and ok flags as nbldpc_decode, bit for bit (the tolerance of every
decoder test here), with 8-bit and with 16-bit messages.  When the code's
message slots do not all fit the fixed array (GF(256) N=384: 196,608 bytes
per slot at 8 bits, twice that at 16), the call runs fewer blocks than the
device keeps resident; those cases check that this clipped grid is really
taken.  It lives in its own file, collected last, so that a run
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


NOALLOC_BYTES = 32 << 20     # NBLDPC_NOALLOC_SCRATCH_BYTES
COUNTER_BYTES = 256


@pytest.mark.parametrize("name,frames,ebn0,bits", [("gf64_n576_dv2_dc4", 700, 1.5, 8),
                                                   ("gf256_n384_dv2_dc6", 400, 2.5, 8),
                                                   ("gf4_n48_dv2_dc4", 1000, 3.0, 8),
                                                   ("gf64_n576_dv2_dc4", 700, 1.5, 16),
                                                   ("gf256_n384_dv2_dc6", 400, 2.5, 16)])
def test_noalloc_matches_workspace_entry_point_twice(name, frames, ebn0, bits):
    w = I.WORKLOADS[name]
    code = I.workload_code(name)
    g = I.make_batch(code, ebn0, 606, frames, device="cuda").gamma
    dec = binding.Decoder.from_code(code)
    if bits != 8:
        dec.set_message_bits(bits)
    if name.startswith("gf256"):
        # resident blocks of this launch shape, from the workspace a large batch needs, against the
        # blocks whose message slots fit the fixed array: the non-allocating call must clip its grid
        v, fpb = dec.tuning()
        slot = fpb * code.nnz * code.q * bits // 8
        resident = (binding.nbldpc_decode_workspace_size(dec.handle, 1 << 20) - COUNTER_BYTES) // slot
        fit = (NOALLOC_BYTES - COUNTER_BYTES) // slot
        assert resident > fit, (resident, fit)
    want = [t.cpu().numpy() for t in dec.decode(g, w["max_iters"], w["early_stop"])]
    for call in range(2):
        sym = torch.full((frames, code.n), 0xAB, dtype=torch.uint8, device="cuda")
        its = torch.full((frames,), -1, dtype=torch.int32, device="cuda")
        ok = torch.full((frames,), 7, dtype=torch.uint8, device="cuda")
        binding.nbldpc_decode_noalloc(dec.handle, g, frames, w["max_iters"], w["early_stop"], sym, its, ok)
        torch.cuda.synchronize()
        got = [sym.cpu().numpy(), its.cpu().numpy(), ok.cpu().numpy()]
        for n, a, b in zip(("symbols", "iterations", "ok"), got, want):
            assert np.array_equal(a, b), f"{name} {bits}-bit: call {call}: {n} differ"
