"""Frame sharding across GPUs (one process per GPU).

Frames are independent (the paper's multicodeword mapping, Sec. 4), so a batch
splits into contiguous frame ranges with no exchange during decoding.  Weak
scaling gives every rank a batch of its own; strong scaling splits one batch
with `shard_range` and, if the caller wants the whole result on every rank,
joins the pieces with `gather_results` (the only collective, after decoding).
"""
from __future__ import annotations

import torch


def shard_range(frames: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of the frames that rank `rank` of `world` decodes (sizes differ by at most one)."""
    if world <= 0 or not 0 <= rank < world or frames < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(frames, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_results(parts: list[torch.Tensor], frames: int, world: int, group=None) -> list[torch.Tensor]:
    """All-gather per-rank output tensors (frames along dim 0) into whole-batch tensors."""
    import torch.distributed as dist
    out = []
    for t in parts:
        sizes = [shard_range(frames, r, world)[1] - shard_range(frames, r, world)[0] for r in range(world)]
        mx = max(sizes)
        pad = torch.zeros((mx,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        pad[: t.shape[0]] = t
        bufs = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(bufs, pad, group=group)
        out.append(torch.cat([b[:s] for b, s in zip(bufs, sizes)], 0))
    return out
