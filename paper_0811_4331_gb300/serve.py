"""Continuous-batching solve server over the C ABI (host-side scheduling only).

Requests -- (gauge field, mass, 1..12 right-hand sides, tolerance) -- arrive
while others are running.  The server keeps, per gauge field, one resident
multigrid hierarchy (the null-vector setup of Sec. 2, done once on the first
request for that field) and, per worker, a private copy of it made by
``mg_retarget``: D(m) = D(0) + m 1 has the same eigenvectors at every mass
(Sec. 1) and P^+ P = 1 (Eq. 2.3), so the coarse operators of any mass are the
cached ones shifted on the diagonal.  A free worker takes the oldest waiting
request and merges into it the waiting requests of the same field, up to 64
right-hand sides, and runs them as one ``mg_solve_masses`` call (a mass per
right-hand side: every kernel of the solve processes the whole batch, and one
coarsest inverse per distinct mass is built in shared launches).  A batch is
admitted while the device bytes of the resident hierarchies, of the batches
in flight (``mg_footprint``) and its own stay within the HBM budget; after a
batch the worker's copy hands its solve buffers back (``mg_release_work``),
so between batches it holds only its hierarchy; each
worker owns a CUDA stream, so batches overlap on the GPU.  All arithmetic
runs in the library's kernels.  A request's result meets its tolerance
whether it is solved alone or in a batch (the batch's outer solve stops when
every right-hand side has converged, so a result solved in a batch can
differ from the one solved alone by the solve's own error, not more).
"""
import collections
import threading
import time

import numpy as np

from . import wilson_mg as wm


class Request:
    __slots__ = ("rid", "field", "mass", "b", "nrhs", "tol", "arrival", "admitted", "done", "x", "stats", "error",
                 "footprint", "event")

    def __init__(self, rid, field, mass, b, tol, arrival):
        self.rid = rid
        self.field = field
        self.mass = mass
        self.b = b
        self.nrhs = b.shape[0] if b.ndim == 7 else 1
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
    """Admit, batch, run and complete solve requests on one GPU.

    fields: {name: (gauge numpy array, dims, setup_mass[, mg_params])}; params:
    the mg_params of fields that bring none; hbm_budget: device bytes for the
    resident hierarchies plus the batches in flight; workers: maximum number
    of concurrent batches (one CUDA stream each); max_batch_rhs: right-hand
    sides per batch (1..64); merge: False serves every request alone; keep_results: False drops each
    request's right-hand sides and solution once its batch is done (its statistics stay), for long streams.
    """

    def __init__(self, fields, params, hbm_budget, workers=4, max_batch_rhs=64, merge=True, keep_results=True):
        import torch
        self.torch = torch
        self.fields = fields
        self.params = params
        self.budget = int(hbm_budget)
        self.max_batch_rhs = int(max_batch_rhs)
        self.merge = merge
        self.keep_results = keep_results
        self.inflight_bytes = 0
        self.inflight = 0
        self.max_inflight = 0
        self.max_inflight_bytes = 0
        self.resident_bytes = 0
        self.batches = []  # sizes (requests, right-hand sides) of the batches run
        self.queue = collections.deque()
        self.lock = threading.Condition()
        self.bases = {}
        self.copies = {}
        self.copy_bytes = {}
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

    @staticmethod
    def nrhs_of(req):
        return req.nrhs

    def footprint(self, field, nrhs):
        return wm.mg_footprint(self.fields[field][1], self.params_of(field), nrhs)

    def submit(self, req):
        req.footprint = self.footprint(req.field, self.nrhs_of(req))
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
        self.copies.clear()
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
                with self.lock:
                    self.resident_bytes += wm.mg_handle_bytes(h)
            return h

    def copy(self, wid, field, stream):
        """Worker wid's private copy of the field's hierarchy (a handle serves one thread at a time)."""
        key = (wid, field)
        h = self.copies.get(key)
        if h is None:
            base = self.base(field)
            with self.base_lock:
                h = wm.mg_retarget(base, self.fields[field][2], stream=stream)
            self.copies[key] = h
            self.copy_bytes[key] = wm.mg_handle_bytes(h)
            with self.lock:
                self.resident_bytes += self.copy_bytes[key]
        return h

    def _settle(self, wid, field, stream):
        """After a batch: the copy hands its solve buffers back (only its hierarchy stays resident;
        the batch's footprint covered the rest) and the resident count follows its real size."""
        key = (wid, field)
        h = self.copies.get(key)
        if h is None:
            return
        wm.mg_release_work(h, stream)
        now = wm.mg_handle_bytes(h)
        with self.lock:
            self.resident_bytes += now - self.copy_bytes[key]
        self.copy_bytes[key] = now

    # ------------------------------------------------------------------ workers
    def _admit(self):
        """The next batch: the oldest waiting request whose footprint fits the free budget, with the
        waiting requests of its field merged in (oldest first) while the batch stays within
        max_batch_rhs right-hand sides and the budget; None when the oldest does not fit."""
        if not self.queue:
            return None
        head = self.queue[0]
        free = self.budget - self.resident_bytes - self.inflight_bytes
        if head.footprint > free:
            if self.inflight == 0:  # the resident hierarchies alone leave it no room: it would wait forever
                self.queue.popleft()
                head.error = "request needs %d bytes, %d of the budget %d are left beside the resident " \
                             "hierarchies" % (head.footprint, free, self.budget)
                head.done = time.perf_counter()
                head.event.set()
            return None
        batch, nrhs = [head], self.nrhs_of(head)
        if self.merge:
            for req in list(self.queue)[1:]:
                k = self.nrhs_of(req)
                if req.field == head.field and nrhs + k <= self.max_batch_rhs and \
                        self.footprint(head.field, nrhs + k) <= free:
                    batch.append(req)
                    nrhs += k
        for req in batch:
            self.queue.remove(req)
        fp = self.footprint(head.field, nrhs)
        for req in batch:
            req.footprint = fp if req is head else 0
        self.inflight_bytes += fp
        self.inflight += 1
        self.max_inflight = max(self.max_inflight, self.inflight)
        self.max_inflight_bytes = max(self.max_inflight_bytes, self.inflight_bytes)
        self.batches.append((len(batch), nrhs))
        return batch

    def _run(self, wid, batch, stream):
        """One batch: every right-hand side of every request in one solve, a mass per right-hand side."""
        field = batch[0].field
        h = self.copy(wid, field, stream)
        bs = [r.b if r.b.ndim == 7 else r.b[None] for r in batch]
        masses = [r.mass for r, b in zip(batch, bs) for _ in range(b.shape[0])]
        B = np.ascontiguousarray(np.concatenate(bs)) if len(bs) > 1 else np.ascontiguousarray(bs[0])
        X = np.zeros_like(B)
        status, st = wm.mg_solve_masses(h, masses, B, X, min(r.tol for r in batch), stream=stream,
                                        raise_on_noconv=False)
        k = 0
        for r, b in zip(batch, bs):
            n = b.shape[0]
            r.x = X[k:k + n] if r.b.ndim == 7 else X[k]
            r.stats = st[k:k + n]
            # a batch that ran out of iterations fails only the requests with a right-hand side
            # above its own tolerance
            if status != wm.MG_OK and (status != wm.MG_ENOCONV or
                                       any(s["true_rel_residual"] > r.tol for s in r.stats)):
                r.error = wm.STATUS_NAMES[status]
            k += n

    def _worker(self, wid):
        torch = self.torch
        stream = self.streams[wid]
        while True:
            with self.lock:
                batch = self._admit()
                while batch is None:
                    if self.stop and not self.queue:
                        return
                    self.lock.wait(0.01)
                    batch = self._admit()
            t = time.perf_counter()
            for req in batch:
                req.admitted = t
            try:
                with torch.cuda.stream(stream):
                    self._run(wid, batch, stream)
            except Exception as e:  # a failed batch must not stop the server
                for req in batch:
                    req.error = str(e)
            self._settle(wid, batch[0].field, stream)
            if not self.keep_results:
                for req in batch:
                    req.b = None
                    req.x = None
            t = time.perf_counter()
            with self.lock:
                for req in batch:
                    req.done = t
                    self.inflight_bytes -= req.footprint
                    self.completed.append(req)
                self.inflight -= 1
                self.lock.notify_all()
            for req in batch:
                req.event.set()


def poisson_arrivals(rate, n, seed):
    """n arrival times (seconds from 0) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def run_stream(server, requests, arrivals):
    """Submit requests at their arrival times (relative to now); wait for all; return latency stats.
    An entry of `requests` may be a function that makes the Request when it arrives (so that a long
    stream does not hold every right-hand side at once)."""
    t0 = time.perf_counter()
    made = []
    for req, ta in zip(requests, arrivals):
        delay = t0 + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        if callable(req):
            req = req()
        made.append(req)
        req.arrival = time.perf_counter()
        server.submit(req)
    requests = made
    for req in requests:
        req.event.wait()
    t1 = time.perf_counter()
    lat = np.array([r.done - r.arrival for r in requests if r.error is None])
    nrhs = sum(r.nrhs for r in requests if r.error is None)
    errors = collections.Counter(r.error[:120] for r in requests if r.error is not None)
    return {"requests": len(requests), "failed": sum(r.error is not None for r in requests),
            "errors": dict(errors.most_common(4)),
            "wall_s": t1 - t0, "solves_per_s": len(lat) / (t1 - t0), "rhs_per_s": nrhs / (t1 - t0),
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None}
