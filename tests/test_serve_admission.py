"""Host-side admission and batching of the solve server, on CPU (no device work).

The server admits the oldest waiting request while the device bytes of the resident hierarchies and of
the batches in flight plus its footprint (mg_footprint, a host computation) stay within the HBM budget,
and merges into it the waiting requests of the same field (oldest first) up to the batch's right-hand-side
limit and the budget; a request larger than the whole budget is refused at submission.  The object is
built without its worker threads and streams, so the real submit/_admit code runs with nothing on a GPU.
"""
import collections
import os
import threading

import numpy as np
import pytest

LIB = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0811_4331_gb300",
                   "libwilsonmg.so")


@pytest.fixture(scope="module")
def serve_mod():
    if not os.path.exists(LIB):
        from paper_0811_4331_gb300 import build
        build.build()
    from paper_0811_4331_gb300 import serve
    return serve


def _server(serve, budget, fields, params, merge=False, max_batch_rhs=64, resident=0):
    s = object.__new__(serve.SolveServer)
    s.fields, s.params, s.budget = fields, params, int(budget)
    s.inflight_bytes = s.inflight = s.max_inflight = s.max_inflight_bytes = 0
    s.resident_bytes = resident
    s.merge, s.max_batch_rhs = merge, max_batch_rhs
    s.batches = []
    s.queue = collections.deque()
    s.lock = threading.Condition()
    return s


def _req(serve, rid, field, nrhs, dims):
    shp = (nrhs,) + (dims[3], dims[2], dims[1], dims[0], 4, 3)
    return serve.Request(rid, field, 0.1, np.zeros(shp if nrhs > 1 else shp[1:], np.complex128), 1e-10, 0.0)


def test_fifo_admission_within_the_budget(serve_mod):
    wm = serve_mod.wm
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], mixed=1)
    dims = (8, 8, 8, 8)
    f1 = wm.mg_footprint(dims, p, 1)
    f4 = wm.mg_footprint(dims, p, 4)
    assert 0 < f1 < f4
    s = _server(serve_mod, f4 + f1, {"a": (None, dims, 0.1)}, p)
    reqs = [_req(serve_mod, 0, "a", 4, dims), _req(serve_mod, 1, "a", 1, dims), _req(serve_mod, 2, "a", 4, dims),
            _req(serve_mod, 3, "a", 1, dims)]
    for r in reqs:
        s.submit(r)
    assert [r.footprint for r in reqs] == [f4, f1, f4, f1]
    (a,) = s._admit()
    (b,) = s._admit()
    assert (a.rid, b.rid) == (0, 1) and s.inflight_bytes == f4 + f1
    assert s._admit() is None            # the head (a 4-RHS request) waits for room
    assert [r.rid for r in s.queue] == [2, 3]  # first in, first out: no request overtakes the head
    s.inflight_bytes -= a.footprint      # request 0 completes
    s.inflight -= 1
    (c,) = s._admit()
    assert c.rid == 2 and s._admit() is None
    assert s.max_inflight == 2 and s.max_inflight_bytes == f4 + f1


def test_request_larger_than_the_budget_is_refused(serve_mod):
    wm = serve_mod.wm
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], mixed=1)
    dims = (8, 8, 8, 8)
    s = _server(serve_mod, wm.mg_footprint(dims, p, 1), {"a": (None, dims, 0.1)}, p)
    r = s.submit(_req(serve_mod, 0, "a", 4, dims))
    assert r.error and "budget" in r.error and r.event.is_set() and not s.queue


def test_same_field_requests_merge_into_one_batch(serve_mod):
    """With merging, the oldest request takes the waiting requests of its field (oldest first) up to the
    right-hand-side limit; other fields keep their place; resident hierarchies count in the budget."""
    wm = serve_mod.wm
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], mixed=1)
    dims = (8, 8, 8, 8)
    fields = {"a": (None, dims, 0.1), "b": (None, dims, 0.1)}
    s = _server(serve_mod, 100 * wm.mg_footprint(dims, p, 64), fields, p, merge=True, max_batch_rhs=8)
    reqs = [_req(serve_mod, 0, "a", 3, dims), _req(serve_mod, 1, "b", 2, dims), _req(serve_mod, 2, "a", 4, dims),
            _req(serve_mod, 3, "a", 2, dims), _req(serve_mod, 4, "a", 1, dims)]
    for r in reqs:
        s.submit(r)
    batch = s._admit()
    assert [r.rid for r in batch] == [0, 2, 4]            # 3 + 4 + 1 = 8 right-hand sides; request 3 would exceed
    assert [r.rid for r in s.queue] == [1, 3]
    assert s.inflight_bytes == wm.mg_footprint(dims, p, 8) and s.batches == [(3, 8)]
    assert sum(r.footprint for r in batch) == s.inflight_bytes
    assert [r.rid for r in s._admit()] == [1]             # the other field's request is next
    # resident hierarchies leave no room: nothing is admitted
    t = _server(serve_mod, wm.mg_footprint(dims, p, 4), fields, p, merge=True,
                resident=wm.mg_footprint(dims, p, 4) - wm.mg_footprint(dims, p, 1) + 1)
    t.submit(_req(serve_mod, 5, "a", 1, dims))
    assert t._admit() is None


def test_stream_makes_requests_on_arrival(serve_mod):
    """run_stream takes functions that make each request when it arrives (a long stream then never holds
    every right-hand side at once); latency and right-hand-side counts come from the made requests."""
    made = []

    class Instant:  # completes every submission at once, with no device work
        def submit(self, req):
            req.done = req.arrival + 0.001
            req.stats = [{}] * req.nrhs
            req.event.set()
            return req

    def factory(i, nrhs):
        def make():
            made.append(i)
            return serve_mod.Request(i, "a", 0.1, np.zeros((nrhs, 1, 1, 1, 1, 4, 3), np.complex128), 1e-10, 0.0)
        return make

    fs = [factory(i, 1 + i % 3) for i in range(6)]
    st = serve_mod.run_stream(Instant(), fs, np.zeros(6))
    assert made == list(range(6))
    assert st["requests"] == 6 and st["failed"] == 0
    assert abs(st["rhs_per_s"] * st["wall_s"] - sum(1 + i % 3 for i in range(6))) < 1e-9
    assert abs(st["p50_s"] - 0.001) < 1e-12
