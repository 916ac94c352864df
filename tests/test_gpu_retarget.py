"""mg_retarget: one null-vector setup serves every mass (D(m) = D(0) + m 1, P^+ P = 1).

Checks: the retargeted coarse stencil is the source's plus (m - m0) on the
diagonal of the self block (exactly, FP64); a solve through the retargeted
handle reaches the true FP64 residual and the unique solution of a fresh
setup at the new mass; the source handle is untouched.
"""
import numpy as np
import pytest

from gpu_util import lattice, rel_err, require_gpu
from oracle import dirac
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mixed", [0, 1])
def test_retarget_shifts_coarse_diagonal_and_solves(mixed):
    wm = require_gpu()
    dims = (8, 8, 4, 8)
    U = inputs.random_gauge(dims, 2)
    m0, m1 = 0.05, -0.15
    p = wm.mg_default_params(n_levels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 6], setup_sweeps=[20, 20],
                             mixed=mixed)
    h0 = wm.mg_setup(U, dims, m0, p)
    h1 = wm.mg_retarget(h0, m1)
    for l in (1, 2):
        A0 = wm.mg_get_coarse_op(h0, l)
        A1 = wm.mg_get_coarse_op(h1, l)
        shift = A1 - A0
        n = A0.shape[-1]
        expect = np.zeros_like(shift)
        expect[0, :, np.arange(n), np.arange(n)] = m1 - m0
        assert np.max(np.abs(shift - expect)) < 1e-14
    b = inputs.gaussian_spinor(dims, 3)
    x1 = np.zeros_like(b)
    wm.mg_solve(h1, b, x1, 1e-10)
    assert np.linalg.norm(b - dirac.wilson_dirac(U, x1, m1)) <= 1e-10 * np.linalg.norm(b)
    hf = wm.mg_setup(U, dims, m1, p)
    xf = np.zeros_like(b)
    wm.mg_solve(hf, b, xf, 1e-10)
    assert rel_err(x1, xf) < 1e-8
    # the source still solves at its own mass
    x0 = np.zeros_like(b)
    wm.mg_solve(h0, b, x0, 1e-10)
    assert np.linalg.norm(b - dirac.wilson_dirac(U, x0, m0)) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("mixed", [0, 1])
def test_batched_retarget_equals_one_by_one(mixed):
    """mg_retarget_batch builds every coarsest inverse in shared launches with the same
    per-matrix arithmetic, so each handle solves bit for bit like its mg_retarget twin."""
    wm = require_gpu()
    dims = (8, 8, 4, 8)
    U = inputs.random_gauge(dims, 5)
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[20], mixed=mixed)
    h0 = wm.mg_setup(U, dims, -0.1, p)
    masses = [0.2, 0.0, -0.05]
    hb = wm.mg_retarget_batch(h0, masses)
    b = inputs.gaussian_spinor(dims, 4)
    for m, h in zip(masses, hb):
        hs = wm.mg_retarget(h0, m)
        xb = np.zeros_like(b)
        xs = np.zeros_like(b)
        _, sb = wm.mg_solve(h, b, xb, 1e-10)
        _, ss = wm.mg_solve(hs, b, xs, 1e-10)
        assert sb[0]["iters"] == ss[0]["iters"]
        assert np.array_equal(xb, xs), m
        assert np.linalg.norm(b - dirac.wilson_dirac(U, xb, m)) <= 1e-10 * np.linalg.norm(b) * 1.001


def test_deferred_coarsest_is_built_on_first_use():
    """defer_coarsest leaves the inverse to the first solve (or to mg_retarget_batch); the
    result is bit for bit the one of a setup that built it at once."""
    wm = require_gpu()
    dims = (8, 8, 4, 8)
    U = inputs.random_gauge(dims, 6)
    b = inputs.gaussian_spinor(dims, 7)
    xs = []
    for defer in (0, 1):
        p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[20], mixed=1,
                                 defer_coarsest=defer)
        h = wm.mg_setup(U, dims, -0.1, p)
        x = np.zeros_like(b)
        wm.mg_solve(h, b, x, 1e-10)
        xs.append(x)
        hb = wm.mg_retarget_batch(h, [-0.1, 0.05])
        xb = np.zeros_like(b)
        wm.mg_solve(hb[0], b, xb, 1e-10)
        assert np.array_equal(xb, x)
    assert np.array_equal(xs[0], xs[1])


@pytest.mark.parametrize("mixed,device", [(1, True), (0, False), (1, False)])
def test_concurrent_solves_equal_one_by_one(mixed, device):
    """mg_solve_many runs independent handles side by side (a thread and stream each); every
    kernel is deterministic, so each handle's x and iteration count are those of mg_solve alone."""
    wm = require_gpu()
    import torch
    dims = (8, 8, 4, 8)
    U = inputs.random_gauge(dims, 8)
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[20], mixed=mixed)
    h0 = wm.mg_setup(U, dims, -0.1, p)
    masses = [0.2, 0.05, 0.0, -0.05]
    B = np.stack([inputs.gaussian_spinor(dims, 20 + r) for r in range(2)])
    want = []
    for m in masses:
        h = wm.mg_retarget(h0, m)
        x = np.zeros_like(B)
        _, st = wm.mg_solve(h, B, x, 1e-10)
        want.append((x, [s["iters"] for s in st]))
    hs = wm.mg_retarget_batch(h0, masses)
    if device:
        bs = [torch.from_numpy(B).cuda() for _ in masses]
        xs = [torch.zeros_like(bs[0]) for _ in masses]
        torch.cuda.synchronize()
        streams = [torch.cuda.Stream() for _ in masses]
    else:
        bs = [B] * len(masses)
        xs = [np.zeros_like(B) for _ in masses]
        streams = None
    status, sts = wm.mg_solve_many(hs, bs, xs, 1e-10, streams=streams)
    assert status == wm.MG_OK
    for m, x, st, (xw, itw) in zip(masses, xs, sts, want):
        x = x.cpu().numpy() if device else x
        assert [s["iters"] for s in st] == itw, m
        assert np.array_equal(x, xw), m
        for r in range(B.shape[0]):
            assert np.linalg.norm(B[r] - dirac.wilson_dirac(U, x[r], m)) <= 1e-10 * np.linalg.norm(B[r]) * 1.001
    with pytest.raises(wm.MgError) as e:
        wm.mg_solve_many([hs[0], hs[0]], [B, B], [np.zeros_like(B), np.zeros_like(B)], 1e-10)
    assert e.value.status == wm.MG_EINVAL and "distinct" in str(e.value)
