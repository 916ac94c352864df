"""Continuous-batching solve server over the C ABI (host-side scheduling only).

Requests -- (gauge field, mass, 1..12 right-hand sides, tolerance) -- arrive
while others are running.  The server keeps, per gauge field, one resident
multigrid hierarchy (the null-vector setup of Sec. 2, done once on the first
request for that field) and serves every request from it through
``mg_retarget``: D(m) = D(0) + m 1 has the same eigenvectors at every mass
(Sec. 1) and P^+ P = 1 (Eq. 2.3), so the coarse operators of another mass are
the cached ones shifted on the diagonal; only the coarsest inverse is
rebuilt.  A request is admitted when a worker is free and the device bytes in
flight plus its own (``mg_footprint``) stay within the HBM budget; each worker
owns a CUDA stream, so admitted requests overlap on the GPU.  All arithmetic
runs in the library's kernels; results do not depend on what else is running
(every reduction is per handle and deterministic).
"""
import collections
import threading
import time

import numpy as np

from . import wilson_mg as wm


class Request:
    __slots__ = ("rid", "field", "mass", "b", "tol", "arrival", "admitted", "done", "x", "stats", "error",
                 "footprint", "event")

    def __init__(self, rid, field, mass, b, tol, arrival):
        self.rid = rid
        self.field = field
        self.mass = mass
        self.b = b
        self.tol = tol
        self.arrival = arrival
        self.admitted = None
        self.done = None
        self.x = None
        self.stats = None
        self.error = None
        self.footprint = 0
        self.event = threading.Event()


class SolveServer:
    """Admit, run and complete solve requests on one GPU.

    fields: {name: (gauge numpy array, dims, setup_mass[, mg_params])}; params:
    the mg_params of fields that bring none; hbm_budget: device bytes the
    in-flight requests may use; workers: maximum number of concurrent requests
    (one CUDA stream each).
    """

    def __init__(self, fields, params, hbm_budget, workers=4):
        import torch
        self.torch = torch
        self.fields = fields
        self.params = params
        self.budget = int(hbm_budget)
        self.inflight_bytes = 0
        self.inflight = 0
        self.max_inflight = 0
        self.max_inflight_bytes = 0
        self.queue = collections.deque()
        self.lock = threading.Condition()
        self.bases = {}
        self.base_lock = threading.Lock()
        self.completed = []
        self.stop = False
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(workers)]
        self.streams = [torch.cuda.Stream() for _ in range(workers)]
        for t in self.workers:
            t.start()

    # ------------------------------------------------------------------ public
    def params_of(self, field):
        f = self.fields[field]
        return f[3] if len(f) > 3 else self.params

    def submit(self, req):
        dims = self.fields[req.field][1]
        nrhs = req.b.shape[0] if req.b.ndim == 7 else 1
        req.footprint = wm.mg_footprint(dims, self.params_of(req.field), nrhs)
        if req.footprint > self.budget:
            req.error = "request needs %d bytes, budget is %d" % (req.footprint, self.budget)
            req.done = time.perf_counter()
            req.event.set()
            return req
        with self.lock:
            self.queue.append(req)
            self.lock.notify_all()
        return req

    def close(self):
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        for t in self.workers:
            t.join()
        self.bases.clear()

    def base(self, field):
        """The resident hierarchy of a gauge field (set up once, on first use)."""
        with self.base_lock:
            h = self.bases.get(field)
            if h is None:
                U, dims, m0 = self.fields[field][:3]
                h = wm.mg_setup(U, dims, m0, self.params_of(field), stream=self.torch.cuda.current_stream())
                self.torch.cuda.synchronize()
                self.bases[field] = h
            return h

    # ------------------------------------------------------------------ workers
    def _admit(self):
        """Next request (FIFO) whose footprint fits the free budget, or None."""
        if not self.queue:
            return None
        req = self.queue[0]
        if self.inflight_bytes + req.footprint > self.budget:
            return None
        self.queue.popleft()
        self.inflight_bytes += req.footprint
        self.inflight += 1
        self.max_inflight = max(self.max_inflight, self.inflight)
        self.max_inflight_bytes = max(self.max_inflight_bytes, self.inflight_bytes)
        return req

    def _worker(self, wid):
        torch = self.torch
        stream = self.streams[wid]
        while True:
            with self.lock:
                req = self._admit()
                while req is None:
                    if self.stop and not self.queue:
                        return
                    self.lock.wait(0.01)
                    req = self._admit()
            req.admitted = time.perf_counter()
            try:
                base = self.base(req.field)
                with torch.cuda.stream(stream):
                    h = wm.mg_retarget(base, req.mass, stream=stream)
                    x = np.zeros_like(req.b)
                    status, st = wm.mg_solve(h, req.b, x, req.tol, stream=stream, raise_on_noconv=False)
                    wm.mg_destroy(h)
                req.x, req.stats = x, st
                if status != wm.MG_OK:
                    req.error = wm.STATUS_NAMES[status]
            except Exception as e:  # a failed request must not stop the server
                req.error = str(e)
            req.done = time.perf_counter()
            with self.lock:
                self.inflight_bytes -= req.footprint
                self.inflight -= 1
                self.completed.append(req)
                self.lock.notify_all()
            req.event.set()


def poisson_arrivals(rate, n, seed):
    """n arrival times (seconds from 0) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def run_stream(server, requests, arrivals):
    """Submit requests at their arrival times (relative to now); wait for all; return latency stats."""
    t0 = time.perf_counter()
    for req, ta in zip(requests, arrivals):
        delay = t0 + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        req.arrival = time.perf_counter()
        server.submit(req)
    for req in requests:
        req.event.wait()
    t1 = time.perf_counter()
    lat = np.array([r.done - r.arrival for r in requests if r.error is None])
    nrhs = sum((r.b.shape[0] if r.b.ndim == 7 else 1) for r in requests if r.error is None)
    return {"requests": len(requests), "failed": sum(r.error is not None for r in requests),
            "wall_s": t1 - t0, "solves_per_s": len(lat) / (t1 - t0), "rhs_per_s": nrhs / (t1 - t0),
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None}
