"""Serving loop on the GPU: requests of mixed codes that overlap in time are
decoded in shared launches, and each one's outputs equal those of decoding it
alone (bit for bit; frames are independent)."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2508_03567_gb300 import binding, inputs as I
from paper_2508_03567_gb300.serving import CudaExecutor, Request, Server

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_each_request_is_the_same_alone_and_in_the_mix():
    codes = [I.workload_code(n) for n in I.MIXED_SET]
    decs = [binding.Decoder.from_code(c) for c in codes]
    ex = CudaExecutor(decs, max_iters=30, streams=3)
    srv = Server(ex, budget_bytes=64 << 20, streams=3)
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(40):
        k = int(rng.integers(len(codes)))
        f = int(rng.integers(1, 25))
        g = I.make_batch(codes[k], I.MIXED_EBN0, 9000 + i, f).gamma.pin_memory()
        reqs.append(Request(rid=i, code=k, gamma=g))
    for wave in (reqs[:10], reqs[10:25], reqs[25:]):
        for r in wave:
            srv.submit(r)
        srv.poll()
    srv.drain()
    assert len(srv.completed) == 40
    assert srv.launches < 40                      # requests shared launches
    assert srv.peak_used <= srv.budget
    for r in reqs:
        alone = decs[r.code].decode(r.gamma.cuda(), 30, 1)
        for got, want in zip((r.sym, r.iters, r.ok), alone):
            assert torch.equal(got, want.cpu()), f"request {r.rid}"
    for r in reqs[::8]:
        ws, wi, wo = oracle.decode(codes[r.code], r.gamma.numpy(), 30, 1, threads=os.cpu_count() or 4)
        assert np.array_equal(r.sym.numpy(), ws) and np.array_equal(r.iters.numpy(), wi)
        assert np.array_equal(r.ok.numpy(), wo)


def test_plain_mode_matches_fixed_iteration_decode():
    code = I.workload_code("gf16_n1024_dv2_dc4")
    dec = binding.Decoder.from_code(code)
    ex = CudaExecutor([dec], max_iters=12, streams=1)
    srv = Server(ex, mode="plain")
    reqs = [Request(rid=i, code=0, gamma=I.make_batch(code, 2.0, 700 + i, 3 + i).gamma.pin_memory())
            for i in range(4)]
    for r in reqs:
        srv.submit(r)
    srv.drain()
    for r in reqs:
        alone = dec.decode(r.gamma.cuda(), 12, 0)
        for got, want in zip((r.sym, r.iters, r.ok), alone):
            assert torch.equal(got, want.cpu())
