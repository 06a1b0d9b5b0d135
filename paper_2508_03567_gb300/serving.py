"""Serving: continuous batching of decode requests of mixed codes on one GPU.

A request is a group of frames of one code (reliabilities in host memory)
that arrives at some time and completes when its decided symbols, iteration
counts and ok flags are back in host memory.  The server

* queues arriving requests and admits them in arrival order while the bytes
  they keep resident on the device (reliabilities, outputs, and the message
  workspace of the launches in flight) stay within a budget;
* launches the admitted requests as one mixed-code persistent decode
  (nbldpc_decode_batch, up to 32 requests per launch) as soon as one of its
  streams is free, so requests that arrive while others are on the GPU run
  in the next launch, concurrently with the launches still in flight;
* retires launches as their completion events fire and releases their bytes.

At low load every request runs alone (short latency); as load grows the
streams stay busy and launches carry more requests (throughput).  Each
frame's result depends only on its own reliabilities (Alg. 2 has no
interaction between frames), so a request decodes to the same outputs alone
or in any mix.

The "plain" mode is the reference point: one fixed-iteration launch per
request, one stream, in arrival order.

The scheduling logic is separate from the device work (an executor object),
so it is tested on the CPU with a fake executor.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import torch


@dataclass
class Request:
    rid: int
    code: int                      # index into the server's decoder list
    gamma: torch.Tensor            # host, [frames, n, q] uint8 (pinned for asynchronous copies)
    t_arrival: float = 0.0
    sym: torch.Tensor | None = None      # host [frames, n] uint8, filled on completion
    iters: torch.Tensor | None = None    # host [frames] int32
    ok: torch.Tensor | None = None       # host [frames] uint8
    t_admit: float = -1.0
    t_launch: float = -1.0
    t_done: float = -1.0

    @property
    def frames(self) -> int:
        return int(self.gamma.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class _Launch:
    requests: list
    token: object
    reserved: int
    stream: int


class Server:
    """Admission, grouping and retirement; device work goes to `executor`.

    executor interface:
      request_bytes(req) -> int          resident device bytes of one request
      launch_bytes(reqs, plain) -> int   workspace of one launch of these requests
      start(reqs, stream_index, plain)   queue copies + decode + copies back, return a token
      done(token) -> bool                completion test (non-blocking)
      finish(token)                      release device buffers of a completed launch
    """

    def __init__(self, executor, budget_bytes: int = 8 << 30, streams: int = 3, max_jobs: int = 32,
                 mode: str = "continuous", clock=time.perf_counter):
        if mode not in ("continuous", "plain"):
            raise ValueError(mode)
        self.ex = executor
        self.budget = int(budget_bytes)
        self.streams = 1 if mode == "plain" else int(streams)
        self.max_jobs = 1 if mode == "plain" else int(max_jobs)
        self.mode = mode
        self.clock = clock
        self.waiting = collections.deque()     # arrived, not admitted
        self.admitted = collections.deque()    # device bytes reserved, not launched
        self.inflight: list[_Launch] = []
        self.used = 0
        self.peak_used = 0
        self.launches = 0
        self.completed: list[Request] = []

    # ---- arrivals
    def submit(self, req: Request, now: float | None = None) -> None:
        req.t_arrival = self.clock() if now is None else now
        self.waiting.append(req)

    # ---- one scheduling round
    def poll(self) -> list[Request]:
        done = []
        now = self.clock()
        still = []
        for ln in self.inflight:
            if self.ex.done(ln.token):
                self.ex.finish(ln.token)
                self.used -= ln.reserved
                for r in ln.requests:
                    r.t_done = now
                done.extend(ln.requests)
            else:
                still.append(ln)
        self.inflight = still
        # admission in arrival order, against the budget (a request larger than
        # the whole budget is admitted alone once nothing else is resident)
        while self.waiting:
            r = self.waiting[0]
            b = self.ex.request_bytes(r)
            if self.used + b > self.budget and (self.used > 0 or self.admitted):
                break
            self.waiting.popleft()
            self.used += b
            r.t_admit = now
            self.admitted.append(r)
        self.peak_used = max(self.peak_used, self.used)
        # launch admitted requests on free streams
        busy = {ln.stream for ln in self.inflight}
        for s in range(self.streams):
            if not self.admitted:
                break
            if s in busy:
                continue
            group = []
            while self.admitted and len(group) < self.max_jobs:
                group.append(self.admitted.popleft())
            wb = self.ex.launch_bytes(group, self.mode == "plain")
            if self.used + wb > self.budget and self.inflight:
                for r in reversed(group):
                    self.admitted.appendleft(r)
                break
            self.used += wb
            self.peak_used = max(self.peak_used, self.used)
            for r in group:
                r.t_launch = now
            token = self.ex.start(group, s, self.mode == "plain")
            self.inflight.append(_Launch(group, token, wb + sum(self.ex.request_bytes(r) for r in group), s))
            # the request bytes were counted at admission; count them once
            self.used -= sum(self.ex.request_bytes(r) for r in group)
            self.launches += 1
            busy.add(s)
        self.completed.extend(done)
        return done

    def idle(self) -> bool:
        return not (self.waiting or self.admitted or self.inflight)

    def drain(self, sleep: float = 0.0) -> None:
        while not self.idle():
            self.poll()
            if sleep:
                time.sleep(sleep)


class CudaExecutor:
    """Device work of the server: copies, nbldpc_decode_batch (or nbldpc_decode in plain mode), copies back."""

    def __init__(self, decoders, max_iters: int, early_stop: int = 1, device="cuda", streams: int = 3):
        from . import binding
        self.b = binding
        self.decs = decoders
        self.max_iters = max_iters
        self.early_stop = early_stop
        self.dev = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(streams)]

    def request_bytes(self, r: Request) -> int:
        d = self.decs[r.code]
        return r.frames * d.n * d.q + r.frames * (d.n + 5)

    def _jobs(self, reqs, bufs):
        return [(self.decs[r.code].handle, g, r.frames, self.max_iters, self.early_stop, s, i, o)
                for r, (g, s, i, o) in zip(reqs, bufs)]

    def launch_bytes(self, reqs, plain: bool = False) -> int:
        if plain:
            return sum(self.b.nbldpc_decode_workspace_size(self.decs[r.code].handle, r.frames) for r in reqs)
        jobs = [(self.decs[r.code].handle, 0, r.frames, self.max_iters, self.early_stop, 0, 0, 0) for r in reqs]
        return self.b.nbldpc_decode_batch_workspace_size(jobs)

    def start(self, reqs, stream_index: int, plain: bool):
        st = self.streams[stream_index % len(self.streams)]
        bufs = []
        with torch.cuda.stream(st):
            for r in reqs:
                d = self.decs[r.code]
                g = torch.empty(r.gamma.shape, dtype=torch.uint8, device=self.dev)
                g.copy_(r.gamma, non_blocking=True)
                bufs.append((g, torch.empty((r.frames, d.n), dtype=torch.uint8, device=self.dev),
                             torch.empty((r.frames,), dtype=torch.int32, device=self.dev),
                             torch.empty((r.frames,), dtype=torch.uint8, device=self.dev)))
            if plain:
                (r,), ((g, s, i, o),) = reqs, bufs
                d = self.decs[r.code]
                ws = torch.empty(self.b.nbldpc_decode_workspace_size(d.handle, r.frames), dtype=torch.uint8,
                                 device=self.dev)
                self.b.nbldpc_decode(d.handle, g, r.frames, self.max_iters, 0, s, i, o, ws, stream=st)
            else:
                jobs = self._jobs(reqs, bufs)
                ws = torch.empty(self.b.nbldpc_decode_batch_workspace_size(jobs), dtype=torch.uint8,
                                 device=self.dev)
                self.b.nbldpc_decode_batch(jobs, ws, stream=st)
            for r, (g, s, i, o) in zip(reqs, bufs):
                r.sym = torch.empty(s.shape, dtype=torch.uint8, pin_memory=True)
                r.iters = torch.empty(i.shape, dtype=torch.int32, pin_memory=True)
                r.ok = torch.empty(o.shape, dtype=torch.uint8, pin_memory=True)
                r.sym.copy_(s, non_blocking=True)
                r.iters.copy_(i, non_blocking=True)
                r.ok.copy_(o, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return (ev, bufs, ws)

    def done(self, token) -> bool:
        return token[0].query()

    def finish(self, token) -> None:
        token[0].synchronize()


def percentile(xs, p: float) -> float:
    if not xs:
        return float("nan")
    s = sorted(xs)
    k = min(len(s) - 1, max(0, int(round(p / 100.0 * (len(s) - 1)))))
    return s[k]
