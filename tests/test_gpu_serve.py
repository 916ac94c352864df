"""Continuous-batching server: overlapping, merged requests give what each request gives alone.

Requests of two gauge fields, several masses and 1-3 right-hand sides are submitted together, so the
queue fills: free workers merge the waiting requests of one field into one solve with a mass per
right-hand side, and batches of the two fields overlap on the GPU (three workers, one stream each).
The HBM budget (the resident hierarchies plus twice the largest request) bounds the bytes in flight.
Each result must meet the true FP64 residual (recomputed by the oracle) and equal the result of the same
request served alone, one request per solve, to 1e-7 relative: both solutions carry a true residual
of at most 1e-10, and the operators of these fields at these masses have condition numbers below 10^3.
"""
import numpy as np
import pytest

from gpu_util import require_gpu
from oracle import dirac
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


def _requests(serve, fields, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        f = ["a", "b"][int(rng.integers(0, 2))]
        dims = fields[f][1]
        nrhs = int(rng.integers(1, 4))
        b = np.stack([inputs.gaussian_spinor(dims, 1000 * seed + 10 * i + r) for r in range(nrhs)])
        mass = float(rng.uniform(-0.2, 0.1))
        reqs.append(serve.Request(i, f, mass, b, 1e-10, 0.0))
    return reqs


def test_batched_mix_equals_alone_and_budget_admission():
    wm = require_gpu()
    import torch
    from paper_0811_4331_gb300 import serve
    fields = {"a": (inputs.random_gauge((4, 4, 4, 4), 1), (4, 4, 4, 4), 0.0),
              "b": (inputs.random_gauge((8, 4, 4, 8), 2), (8, 4, 4, 8), 0.0)}
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[20], mixed=1)
    one = max(wm.mg_footprint(fields[f][1], p, 3) for f in fields)
    srv = serve.SolveServer(fields, p, hbm_budget=1 << 62, workers=3)
    for f in fields:  # the resident hierarchies: one per field and a private copy per worker
        for w in range(3):
            srv.copy(w, f, srv.streams[w])
    torch.cuda.synchronize()
    assert srv.resident_bytes > 0
    srv.budget = srv.resident_bytes + 2 * one
    reqs = _requests(serve, fields, 16, 1)
    stats = serve.run_stream(srv, reqs, np.zeros(len(reqs)))
    srv.close()
    assert stats["failed"] == 0
    assert srv.max_inflight >= 2                                   # batches overlapped
    assert max(n for n, _ in srv.batches) >= 2                     # requests were merged
    assert srv.max_inflight_bytes <= 2 * one                       # the budget was never exceeded
    for r in reqs:
        U, dims, _ = fields[r.field]
        for k in range(r.b.shape[0]):
            res = np.linalg.norm(r.b[k] - dirac.wilson_dirac(U, r.x[k], r.mass)) / np.linalg.norm(r.b[k])
            assert res <= 1e-10, (r.rid, k, res)
    # the same requests one at a time, one request per solve
    alone = serve.SolveServer(fields, p, hbm_budget=1 << 62, workers=1, merge=False)
    again = _requests(serve, fields, 16, 1)
    for r in again:
        alone.submit(r)
        r.event.wait()
    alone.close()
    assert all(n == 1 for n, _ in alone.batches)
    for r, q in zip(reqs, again):
        assert r.error is None and q.error is None
        rel = np.linalg.norm(r.x - q.x) / np.linalg.norm(q.x)
        assert rel <= 1e-7, (r.rid, rel)


def test_resident_hierarchies_beyond_the_budget_refuse_instead_of_waiting():
    wm = require_gpu()
    from paper_0811_4331_gb300 import serve
    fields = {"a": (inputs.random_gauge((4, 4, 4, 4), 1), (4, 4, 4, 4), 0.0)}
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[5], mixed=1)
    one = wm.mg_footprint((4, 4, 4, 4), p, 1)
    srv = serve.SolveServer(fields, p, hbm_budget=one, workers=1)
    srv.base("a")
    b = inputs.gaussian_spinor((4, 4, 4, 4), 3)
    r = srv.submit(serve.Request(0, "a", 0.05, b, 1e-10, 0.0))
    assert r.event.wait(30)
    srv.close()
    assert r.error and "resident" in r.error
