"""Serving: continuous batching of decode requests of mixed codes on one GPU.

A request is a group of frames of one code (reliabilities in host memory)
that arrives at some time and completes when its decided symbols, iteration
counts and ok flags are back in host memory.  The scheduler is native
(nbldpc_server_* in the C ABI): it queues arriving requests, admits them in
arrival order while the device bytes they keep resident (reliabilities,
outputs, and the workspace of the launches in flight) fit a budget, launches
the admitted requests as one mixed-code persistent decode (up to 32 per
launch) as soon as one of its streams is free, and retires launches as their
completion events fire.  Requests arriving while others are on the GPU run in
the next launch, concurrently with the launches still in flight.

At low load every request runs alone (short latency); as load grows the
streams stay busy and launches carry more requests (throughput).  Each
frame's result depends only on its own reliabilities (Alg. 2 has no
interaction between frames), so a request decodes to the same outputs alone
or in any mix.  "Plain" mode is the reference point: one fixed-iteration
launch per request, one stream, in arrival order.

This module is the Python face of that scheduler: `Server` with the
library's CUDA executor (`CudaExecutor` names the decoders and iteration
settings), or with any Python object that implements the executor calls
(used on the CPU with a fake executor to test the scheduling logic).
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass

import torch

from . import binding


@dataclass
class Request:
    rid: int
    code: int                      # index into the executor's decoder list
    gamma: torch.Tensor            # host, [frames, n, q] uint8 (pinned for asynchronous copies)
    t_arrival: float = 0.0
    sym: torch.Tensor | None = None      # host [frames, n] uint8, written by completion
    iters: torch.Tensor | None = None    # host [frames] int32
    ok: torch.Tensor | None = None       # host [frames] uint8
    t_launch: float = -1.0               # set by Python executors' start (the native executor does not report it)
    t_done: float = -1.0

    @property
    def frames(self) -> int:
        return int(self.gamma.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class CudaExecutor:
    """The library's CUDA executor for a Server: copies in, nbldpc_decode_batch (plain mode: one
    fixed-iteration nbldpc_decode per request), copies out, one event per launch, device buffers from
    the stream-ordered allocator.  Holds the decoders that Request.code indexes and the iteration
    settings of every request."""

    def __init__(self, decoders, max_iters: int, early_stop: int = 1, device="cuda", streams: int = 3):
        self.decs = decoders
        self.max_iters = int(max_iters)
        self.early_stop = int(early_stop)
        self.dev = torch.device(device)
        self.streams = int(streams)


class Server:
    """Native scheduler; device work by `executor` (a CudaExecutor, or a Python object with
    request_bytes(req), launch_bytes(reqs, plain), start(reqs, stream, plain) -> token,
    done(token) -> bool and finish(token)).  An exception raised by a Python executor is
    re-raised by the submit or poll call that ran it; the server should then be discarded."""

    POLL_BATCH = 256

    def __init__(self, executor, budget_bytes: int = 8 << 30, streams: int = 3, max_jobs: int = 32,
                 mode: str = "continuous", clock=time.perf_counter):
        if mode not in ("continuous", "plain"):
            raise ValueError(mode)
        self.budget = int(budget_bytes)
        self.mode = mode
        self.clock = clock
        self.completed: list[Request] = []
        self._ex = executor
        self._native = isinstance(executor, CudaExecutor)
        self._tags: dict[int, Request] = {}     # user tag -> request (submitted, not completed)
        self._ids: dict[int, Request] = {}      # server id -> request
        self._next_tag = 1
        self._tokens: dict[int, object] = {}   # Python executor tokens by native token
        self._next_token = 1
        self._pending: BaseException | None = None   # raised by a Python executor inside a native call
        self._h = ctypes.c_void_p()
        L = binding.lib()
        plain = 1 if mode == "plain" else 0
        if self._native:
            if executor.dev.index is not None:        # the server works on the current device
                torch.cuda.set_device(executor.dev.index)
            st = L.nbldpc_server_create(self.budget, int(streams), int(max_jobs), plain, ctypes.byref(self._h))
        else:
            self._callbacks = self._make_callbacks()
            exs = binding.nbldpc_server_executor(None, *self._callbacks)
            st = L.nbldpc_server_create_custom(ctypes.byref(exs), self.budget, int(streams), int(max_jobs), plain,
                                               ctypes.byref(self._h))
        binding._check(st, "nbldpc_server_create")
        self._buf = (ctypes.c_uint64 * self.POLL_BATCH)()

    # ---- Python executors behind the native scheduler
    # An exception must not unwind through C: a callback records it and returns a
    # neutral value (byte counts) or an error status (launch calls); the Python call
    # that entered the native scheduler re-raises it (_raise_pending).
    def _make_callbacks(self):
        ex = self._ex

        def reqs_of(arr, n):
            return [self._tags[arr[i].contents.user] for i in range(n)]

        def guarded(fn, failed):
            def cb(*args):
                try:
                    return fn(*args)
                except BaseException as e:  # noqa: BLE001 - re-raised after the native call
                    if self._pending is None:
                        self._pending = e
                    return failed
            return cb

        def request_bytes(_ctx, rp):
            return int(ex.request_bytes(self._tags[rp.contents.user]))

        def launch_bytes(_ctx, arr, n, plain):
            return int(ex.launch_bytes(reqs_of(arr, n), bool(plain)))

        def start(_ctx, arr, n, stream, plain, tok):
            reqs = reqs_of(arr, n)
            now = self.clock()
            for r in reqs:
                r.t_launch = now
            k = self._next_token
            self._next_token += 1
            self._tokens[k] = ex.start(reqs, int(stream), bool(plain))
            tok[0] = k
            return binding.NBLDPC_OK

        def done(_ctx, k):
            return 1 if ex.done(self._tokens[k]) else 0

        def finish(_ctx, k):
            ex.finish(self._tokens.pop(k))
            return binding.NBLDPC_OK

        err = binding.NBLDPC_ERR_ARG
        return (binding.REQUEST_BYTES_FN(guarded(request_bytes, 0)),
                binding.LAUNCH_BYTES_FN(guarded(launch_bytes, 0)),
                binding.START_FN(guarded(start, err)), binding.TOKEN_FN(guarded(done, err)),
                binding.TOKEN_FN(guarded(finish, err)))

    def _raise_pending(self) -> None:
        if self._pending is not None:
            e, self._pending = self._pending, None
            raise e

    # ---- arrivals
    def submit(self, req: Request, now: float | None = None) -> None:
        req.t_arrival = self.clock() if now is None else now
        tag = self._next_tag
        self._next_tag += 1
        r = binding.nbldpc_request()
        r.frames = req.frames
        r.user = tag
        if self._native:
            d = self._ex.decs[req.code]
            if not req.gamma.is_contiguous():
                raise ValueError("request reliabilities must be contiguous host memory")
            req.sym = torch.empty((req.frames, d.n), dtype=torch.uint8, pin_memory=True)
            req.iters = torch.empty((req.frames,), dtype=torch.int32, pin_memory=True)
            req.ok = torch.empty((req.frames,), dtype=torch.uint8, pin_memory=True)
            r.code = d.handle
            r.gamma_host = req.gamma.data_ptr()
            r.max_iters = self._ex.max_iters
            r.early_stop = self._ex.early_stop
            r.out_sym_host = req.sym.data_ptr()
            r.out_iters_host = req.iters.data_ptr()
            r.out_ok_host = req.ok.data_ptr()
        self._tags[tag] = req
        rid = ctypes.c_uint64()
        st = binding.lib().nbldpc_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid))
        self._raise_pending()
        binding._check(st, "nbldpc_server_submit")
        self._ids[rid.value] = req
        req._tag = tag

    # ---- one scheduling round
    def poll(self) -> list[Request]:
        done = []
        L = binding.lib()
        n = ctypes.c_int()
        while True:
            st = L.nbldpc_server_poll(self._h, self._buf, self.POLL_BATCH, ctypes.byref(n))
            self._raise_pending()
            binding._check(st, "nbldpc_server_poll")
            now = self.clock() if n.value else 0.0
            for i in range(n.value):
                req = self._ids.pop(self._buf[i])
                self._tags.pop(req._tag, None)
                req.t_done = now
                done.append(req)
            if n.value < self.POLL_BATCH:
                break
        self.completed.extend(done)
        return done

    def stats(self) -> binding.nbldpc_server_stats:
        st = binding.nbldpc_server_stats()
        binding._check(binding.lib().nbldpc_server_stats_get(self._h, ctypes.byref(st)), "nbldpc_server_stats_get")
        return st

    @property
    def used(self) -> int:
        return int(self.stats().used_bytes)

    @property
    def peak_used(self) -> int:
        return int(self.stats().peak_bytes)

    @property
    def launches(self) -> int:
        return int(self.stats().launches)

    def idle(self) -> bool:
        st = self.stats()
        return st.submitted == st.completed

    def drain(self, sleep: float = 0.0) -> None:
        while not self.idle():
            self.poll()
            if sleep:
                time.sleep(sleep)

    def close(self) -> None:
        if self._h:
            binding.lib().nbldpc_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def percentile(xs, p: float) -> float:
    if not xs:
        return float("nan")
    s = sorted(xs)
    k = min(len(s) - 1, max(0, int(round(p / 100.0 * (len(s) - 1)))))
    return s[k]
