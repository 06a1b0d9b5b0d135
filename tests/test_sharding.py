"""Frame sharding over ranks (world size 2, gloo, CPU): each rank decodes its
contiguous share with the CPU oracle and the gathered result equals the
whole-batch decode."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2508_03567_gb300 import inputs as I
from paper_2508_03567_gb300.sharding import gather_results, shard_range


def test_shard_range_partitions():
    for frames in (0, 1, 5, 196608, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard_range(frames, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == frames
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [h - l for l, h in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    code = I.workload_code("gf16_n1024_dv2_dc4")
    frames = 7
    g = I.make_batch(code, 1.5, 123, frames).gamma.numpy()
    lo, hi = shard_range(frames, rank, world)
    sym, its, ok = oracle.decode(code, g[lo:hi], 30, 1)
    parts = [torch.from_numpy(sym), torch.from_numpy(its), torch.from_numpy(ok)]
    full = gather_results(parts, frames, world)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)          # max-over-ranks timing reduction
    if rank == 0:
        np.savez(result_path, sym=full[0].numpy(), its=full[1].numpy(), ok=full[2].numpy(),
                 tmax=t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_match_single_process(tmp_path, oracle_lib):
    path = str(tmp_path / "r.npz")
    mp.start_processes(_worker, args=(2, _free_port(), path), nprocs=2, start_method="spawn")
    r = np.load(path)
    code = I.workload_code("gf16_n1024_dv2_dc4")
    g = I.make_batch(code, 1.5, 123, 7).gamma.numpy()
    sym, its, ok = oracle_lib.decode(code, g, 30, 1)
    assert np.array_equal(r["sym"], sym) and np.array_equal(r["its"], its) and np.array_equal(r["ok"], ok)
    assert r["tmax"][0] == 2.0
