"""Serving dispatcher host logic (CPU): admission by slots and memory budget,
arrival order, and a failing request reported without stopping the others.
The device work is replaced by a fake executor; no GPU is touched."""

import threading
import time

import numpy as np
import pytest

serve = pytest.importorskip("paper_2503_21176_gb300.serve")


class FakeServer(serve.Server):
    """The dispatcher of Server with a host-side executor: each request sleeps,
    records the memory reserved while it runs, and fails when asked to."""

    def __init__(self, max_inflight, budget, fail=()):
        self.max_inflight = max_inflight
        self.budget = budget
        self.streams = [None] * max_inflight
        self._free_slots = list(range(max_inflight))
        self._lock = threading.Lock()
        self._reserved = 0
        self.fail = set(fail)
        self.seen_reserved = []
        self.running = 0
        self.max_running = 0
        self.mu = threading.Lock()

    def _execute(self, req, slot, t0, t_admit):
        with self.mu:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.seen_reserved.append(self._reserved)
        time.sleep(0.01)
        with self.mu:
            self.running -= 1
        if req.rid in self.fail:
            raise RuntimeError(f"malformed request {req.rid}")
        n = req.n_atoms
        return serve.Result(req.rid, req.kind, n, np.zeros(n), np.zeros((n, 3)), req.R.copy(),
                            {"total": 0.0}, t0 + req.arrival, t_admit, time.perf_counter(),
                            {"create": 0.1})


def _requests(sizes):
    out = []
    for k, n in enumerate(sizes):
        R = np.zeros((n, 3))
        z = np.zeros(n)
        out.append(serve.Request(k, "qeq", R, np.array([20.0, 20.0, 20.0]), z, z, z + 0.5, z + 1.0,
                                 (16, 16, 16), arrival=0.001 * k))
    return out


def test_all_requests_served_within_the_slots():
    reqs = _requests([30, 60, 90, 120, 30, 60])
    srv = FakeServer(max_inflight=2, budget=1 << 40)
    res, stats = srv.serve(reqs, realtime=False)
    assert [r.rid for r in res] == list(range(6))
    assert stats["requests"] == 6 and stats["failed"] == 0
    assert srv.max_running <= 2 and stats["max_concurrent"] <= 2


def test_memory_budget_limits_concurrency():
    reqs = _requests([300] * 4)
    one = max(serve.estimate_device_bytes(r) for r in reqs)
    srv = FakeServer(max_inflight=4, budget=one)  # room for one request at a time
    res, stats = srv.serve(reqs, realtime=False)
    assert stats["requests"] == 4 and srv.max_running == 1
    assert max(srv.seen_reserved) <= one
    with pytest.raises(MemoryError):
        FakeServer(max_inflight=2, budget=1024).serve(reqs[:1])


def test_a_failing_request_is_reported_and_the_rest_complete():
    reqs = _requests([30, 60, 90, 120])
    res, stats = FakeServer(max_inflight=2, budget=1 << 40, fail={1}).serve(reqs, realtime=False)
    assert stats["requests"] == 4 and stats["failed"] == 1
    assert res[1].error == "RuntimeError: malformed request 1" and res[1].q is None
    assert all(r.error is None and r.q is not None for k, r in enumerate(res) if k != 1)
