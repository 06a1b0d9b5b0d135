"""Scheduling logic of the serving loop, on the CPU with a fake executor
(arrival order, memory budget, grouping, streams, plain mode)."""
import numpy as np
import torch

from paper_2508_03567_gb300.serving import Request, Server, percentile


class FakeExecutor:
    """Completes a launch after `delay` polls; records what it was asked to do and which launches are
    outstanding (started, not finished) with their stream and resident bytes."""

    def __init__(self, req_bytes=100, ws_bytes=50, delay=2):
        self.req_bytes, self.ws_bytes, self.delay = req_bytes, ws_bytes, delay
        self.starts = []
        self.polls = {}
        self.active = {}

    def request_bytes(self, r):
        return self.req_bytes * r.frames

    def launch_bytes(self, reqs, plain=False):
        return self.ws_bytes

    def start(self, reqs, stream, plain):
        tok = len(self.starts)
        self.starts.append(([r.rid for r in reqs], stream, plain))
        self.polls[tok] = 0
        self.active[tok] = (stream, self.ws_bytes + sum(self.request_bytes(r) for r in reqs))
        for r in reqs:
            r.sym = torch.zeros((r.frames, 1), dtype=torch.uint8)
        return tok

    def done(self, tok):
        self.polls[tok] += 1
        return self.polls[tok] > self.delay

    def finish(self, tok):
        del self.active[tok]


def req(i, frames=1):
    return Request(rid=i, code=0, gamma=torch.zeros((frames, 1, 2), dtype=torch.uint8))


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


def test_budget_is_never_exceeded_and_order_is_kept():
    ex = FakeExecutor(req_bytes=100, ws_bytes=50)
    srv = Server(ex, budget_bytes=1000, streams=2, max_jobs=4, clock=Clock())
    rng = np.random.default_rng(0)
    for i in range(60):
        srv.submit(req(i, int(rng.integers(1, 4))))
        srv.poll()
        # the accounted bytes cover every launch in flight (its workspace and its requests) and
        # never pass the budget
        assert sum(b for _, b in ex.active.values()) <= srv.used <= srv.budget
    srv.drain()
    assert srv.peak_used <= srv.budget
    assert srv.used == 0 and not ex.active                   # everything released
    launched = [rid for rids, _, _ in ex.starts for rid in rids]
    assert launched == list(range(60))                       # arrival order
    assert all(len(rids) <= 4 for rids, _, _ in ex.starts)   # group size limit
    assert sorted(r.rid for r in srv.completed) == list(range(60))
    assert all(r.t_arrival <= r.t_launch <= r.t_done for r in srv.completed)


def test_streams_are_not_oversubscribed():
    ex = FakeExecutor(delay=5)
    srv = Server(ex, budget_bytes=1 << 30, streams=3, max_jobs=2, clock=Clock())
    for i in range(20):
        srv.submit(req(i))
    for _ in range(200):
        srv.poll()
        streams = [st for st, _ in ex.active.values()]
        assert len(streams) <= 3 and len(set(streams)) == len(streams)
        if srv.idle():
            break
    assert srv.idle()


def test_requests_arriving_during_a_launch_join_the_next_one():
    ex = FakeExecutor(delay=3)
    srv = Server(ex, budget_bytes=1 << 30, streams=1, max_jobs=32, clock=Clock())
    srv.submit(req(0))
    srv.poll()                                  # launches request 0 alone
    for i in range(1, 6):                       # arrive while request 0 is on the GPU
        srv.submit(req(i))
    srv.drain()
    assert ex.starts[0][0] == [0]
    assert ex.starts[1][0] == [1, 2, 3, 4, 5]   # batched while the GPU was busy


def test_oversized_request_runs_alone():
    ex = FakeExecutor(req_bytes=100, ws_bytes=10)
    srv = Server(ex, budget_bytes=250, streams=2, clock=Clock())
    srv.submit(req(0, 1))
    srv.submit(req(1, 9))                        # 900 bytes > budget
    srv.submit(req(2, 1))
    srv.drain()
    assert [rids for rids, _, _ in ex.starts] == [[0], [1], [2]]


def test_plain_mode_serializes_single_requests():
    ex = FakeExecutor(delay=1)
    srv = Server(ex, budget_bytes=1 << 30, streams=4, max_jobs=32, mode="plain", clock=Clock())
    for i in range(7):
        srv.submit(req(i))
    srv.drain()
    assert [rids for rids, _, _ in ex.starts] == [[i] for i in range(7)]
    assert all(s == 0 and plain for _, s, plain in ex.starts)


def test_percentile():
    xs = list(range(101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99 and percentile(xs, 0) == 0


def test_executor_errors_surface_in_python():
    """An exception inside the Python executor is raised by the call that drove the scheduler."""
    class Broken(FakeExecutor):
        def start(self, reqs, stream, plain):
            raise RuntimeError("device lost")

    srv = Server(Broken(), budget_bytes=1 << 20, streams=1, clock=Clock())
    srv.submit(req(0))
    try:
        srv.poll()
    except RuntimeError as e:
        assert "device lost" in str(e)
    else:
        raise AssertionError("the executor's exception was swallowed")

    class BadBytes(FakeExecutor):
        def request_bytes(self, r):
            raise ValueError("no size")

    srv2 = Server(BadBytes(), budget_bytes=1 << 20, streams=1, clock=Clock())
    try:
        srv2.submit(req(1))
    except ValueError as e:
        assert "no size" in str(e)
    else:
        raise AssertionError("the executor's exception was swallowed")
