"""Host logic of the serving loop and of the footprint it admits by (no GPU needed): FIFO
admission by HBM footprint, releasing an idle worker's cached workspace only when that is what
blocks the queue head, the reservation arithmetic, the latency summary, and the closed-form
structure of pt_ptim_footprint (pure host arithmetic in the C library)."""
import collections
import types

import numpy as np
import pytest

from paper_2501_03061_gb300 import synth


def server_stub(budget, workers):
    from paper_2501_03061_gb300.serve import Server
    s = object.__new__(Server)  # the scheduling state only; no device, threads or contexts
    s.budget = budget
    s.workers = workers
    s.queue = collections.deque()
    s.sessions = {}
    return s


def worker(held=0, reserved=0, busy=False):
    return types.SimpleNamespace(held=held, reserved=reserved, busy=busy)


def request(footprint, session=None):
    return types.SimpleNamespace(footprint=footprint, session=session)


def test_admits_queue_head_on_the_worker_with_the_largest_cache():
    a, b = worker(held=10), worker(held=30)
    s = server_stub(100, [a, b])
    s.queue.append((request(40), None))
    w, trim = s._pick()
    assert w is b and trim is None  # 40 + max(10, 0) = 50 <= 100 using b's cache
    assert s._reserved() == 40


def test_empty_queue_or_no_free_worker_admits_nothing():
    s = server_stub(100, [worker(busy=True, reserved=50)])
    assert s._pick() == (None, None)
    s.queue.append((request(10), None))
    assert s._pick() == (None, None)


def test_trims_an_idle_cache_only_when_it_blocks_the_head():
    busy = worker(busy=True, reserved=50)
    big_idle, small_idle = worker(held=40), worker(held=20)
    s = server_stub(100, [busy, big_idle, small_idle])
    s.queue.append((request(45), None))
    # reserved now 50 + 40 + 20 = 110; on big_idle: 110 - 40 + max(40, 45) = 115 > 100 -> release
    # the cache of the other idle worker (small_idle), then the head fits on big_idle
    w, trim = s._pick()
    assert w is None and trim is small_idle
    small_idle.held = 0
    w, trim = s._pick()
    assert w is big_idle and trim is None


def test_waits_while_running_requests_hold_the_memory():
    s = server_stub(100, [worker(busy=True, reserved=70), worker(held=0)])
    s.queue.append((request(40), None))
    assert s._pick() == (None, None)  # 70 + 40 > 100 and no idle cache to release
    s.workers[0].busy = False
    s.workers[0].reserved = 0
    s.workers[0].held = 5
    w, trim = s._pick()
    assert w is s.workers[0]  # FIFO head admitted once memory is free


def test_reservation_counts_the_larger_of_cache_and_reservation():
    s = server_stub(10 ** 9, [worker(held=30, reserved=10), worker(held=5, reserved=50), worker()])
    assert s._reserved() == 30 + 50


def test_latency_summary_percentiles():
    from paper_2501_03061_gb300.serve import latency_summary
    reqs = [types.SimpleNamespace(latency=float(i), error=None, t_end=1.0) for i in range(1, 101)]
    reqs.append(types.SimpleNamespace(latency=1e9, error="failed", t_end=1.0))  # errors excluded
    out = latency_summary(reqs)
    assert out["count"] == 100
    assert out["p50_s"] == pytest.approx(np.percentile(np.arange(1, 101), 50))
    assert out["p99_s"] == pytest.approx(np.percentile(np.arange(1, 101), 99))
    assert out["max_s"] == 100.0
    assert latency_summary([]) == {"count": 0}


def test_footprint_structure():
    """pt_ptim_footprint: the Anderson ring adds two orbital blocks and two N x N matrices per
    history entry, FP64 needs more than FP32, the footprint grows with N, and the 64^3 FP32
    exchange's four scratch slots of B x B pair fields are in it."""
    from paper_2501_03061_gb300 import api
    cell = synth.cubic(48, 15.0)
    ng = 48 ** 3
    for N in (32, 200):
        d = api.ptim_footprint(N, cell, "fp32", 20) - api.ptim_footprint(N, cell, "fp32", 10)
        assert d == 2 * 10 * (N * ng * 8 + N * N * 16)
        assert api.ptim_footprint(N, cell, "fp64", 20) > api.ptim_footprint(N, cell, "fp32", 20)
    assert api.ptim_footprint(200, cell, "fp32", 20) > api.ptim_footprint(32, cell, "fp32", 20)
    c64 = synth.cubic(64, 20.5)
    f = api.ptim_footprint(320, c64, "fp32", 20)
    assert f >= (12 + 40) * 320 * 64 ** 3 * 8 + 4 * 16 * 16 * 64 ** 3 * 8
    assert f < 60 * 2 ** 30


def test_a_failing_request_is_recorded_and_frees_its_worker():
    """_run: an exception inside a request becomes the request's error; the worker is released with
    its workspace size re-read, the request is completed and its future resolved (no device: the
    worker's stream is None and the context is a stub)."""
    import threading
    from concurrent.futures import Future

    from paper_2501_03061_gb300.serve import Request

    s = server_stub(100, [])
    s.cv = threading.Condition()
    s.completed = []
    w = types.SimpleNamespace(held=0, reserved=40, busy=True, stream=None,
                              ctx=types.SimpleNamespace(workspace_bytes=lambda: 17))
    s.workers = [w]

    def boom(worker, req):
        raise ValueError("PT_INVALID_ARG: phi holds 1536 elements where the call addresses 1152")

    s._execute = boom
    req = Request(phi=np.zeros((1, 2, 2, 2), np.complex64), sigma=None, occ=None, vloc=None,
                  cell=synth.cubic(8, 5.0), kernel={})
    fut = Future()
    s._run(w, req, fut)
    assert fut.done() and fut.result() is req
    assert "PT_INVALID_ARG" in req.error and req.result is None
    assert req.t_end >= req.t_start > 0
    assert (w.busy, w.reserved, w.held) == (False, 0, 17)
    assert s.completed == [req]


def test_open_session_state_counts_against_the_budget():
    a = worker()
    s = server_stub(100, [a])
    s.sessions[0] = {"bytes": 70, "busy": False}
    s.queue.append((request(40), None))
    assert s._reserved() == 70
    w, trim = s._pick()
    assert w is None and trim is None  # 70 resident + 40 > 100
    s.sessions.clear()
    w, trim = s._pick()
    assert w is a


def test_session_requests_run_one_at_a_time_in_order():
    a, b = worker(), worker()
    s = server_stub(1000, [a, b])
    s.sessions[3] = {"bytes": 10, "busy": True}  # its previous request is still running
    s.queue.append((request(20, session=3), None))
    s.queue.append((request(20), None))
    w, trim = s._pick()
    assert w is None and trim is None  # the head waits for its session; FIFO keeps the rest behind it
    s.sessions[3]["busy"] = False
    w, trim = s._pick()
    assert w is not None
