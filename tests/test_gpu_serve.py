"""Continuous-batching server: overlapping requests give the same results as each request alone.

Requests of two gauge fields, several masses and 1-3 right-hand sides arrive
as a Poisson stream and overlap on the GPU (three workers, one stream each);
the HBM budget (twice the largest request) bounds the bytes in flight.  Each result must meet the true
FP64 residual (recomputed by the oracle) and equal, bit for bit, the result of
the same request served alone (every reduction is per handle and
deterministic, so the mix cannot change a result).
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


def test_mix_equals_alone_and_budget_admission():
    wm = require_gpu()
    from paper_0811_4331_gb300 import serve
    fields = {"a": (inputs.random_gauge((4, 4, 4, 4), 1), (4, 4, 4, 4), 0.0),
              "b": (inputs.random_gauge((8, 4, 4, 8), 2), (8, 4, 4, 8), 0.0)}
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[20], mixed=1)
    one = max(wm.mg_footprint(fields[f][1], p, 3) for f in fields)
    srv = serve.SolveServer(fields, p, hbm_budget=2 * one, workers=3)
    reqs = _requests(serve, fields, 12, 1)
    stats = serve.run_stream(srv, reqs, serve.poisson_arrivals(200.0, len(reqs), 4))
    srv.close()
    assert stats["failed"] == 0
    assert srv.max_inflight >= 2                      # requests overlapped
    assert srv.max_inflight_bytes <= 2 * one          # the budget was never exceeded
    for r in reqs:
        U, dims, _ = fields[r.field]
        for k in range(r.b.shape[0]):
            res = np.linalg.norm(r.b[k] - dirac.wilson_dirac(U, r.x[k], r.mass)) / np.linalg.norm(r.b[k])
            assert res <= 1e-10, (r.rid, k, res)
    # the same requests one at a time
    alone = serve.SolveServer(fields, p, hbm_budget=10 * one, workers=1)
    again = _requests(serve, fields, 12, 1)
    for r in again:
        alone.submit(r)
        r.event.wait()
    alone.close()
    for r, q in zip(reqs, again):
        assert r.error is None and q.error is None
        assert np.array_equal(r.x, q.x), r.rid
