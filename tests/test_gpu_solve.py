"""GPU MG-GCR solves, checked against the true FP64 residual (recomputed by the oracle) and
against the unique solution x = D^-1 b (dense LU where the lattice is small).

The solution of D x = b is unique (Sec. 1: Re(lambda) > 0 at these masses), so
the multigrid internals (precision, batching) may change iteration counts but
not x.  Tolerance on x: ||x - x_LU|| / ||x_LU|| <= 1e-8 (residual 1e-10 times
the condition number of these small systems).
"""
import numpy as np
import pytest
import scipy.linalg

from gpu_util import lattice, rel_err, require_gpu, torch
from oracle import dirac
from oracle import multigrid as mg
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


def _true_rel(U, mass, x, b):
    return float(np.linalg.norm(b - dirac.wilson_dirac(U, x, mass)) / np.linalg.norm(b))


def _small_workload():
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 0)
    b = inputs.gaussian_spinor(dims, 1)
    starts = [np.stack(inputs.null_vector_starts(lattice(dims), 12, 8, 2)).reshape(8, -1, 12)]
    return dims, U, b, starts


@pytest.fixture(scope="module")
def lu_small():
    dims, U, b, starts = _small_workload()
    D = dirac.dense_matrix(lambda y: dirac.wilson_dirac(U, y, 0.1), lattice(dims) + (4, 3))
    return scipy.linalg.lu_factor(D)


@pytest.mark.parametrize("mixed,fine", [(0, 0), (1, 2), (1, 3), (1, 1)])
def test_small_two_level_solve(mixed, fine, lu_small):
    """4^4, U = exp(0.3 i H), m = 0.1, 2^4 blocks, Nv = 8, 10 setup sweeps, tol 1e-10."""
    wm = require_gpu()
    dims, U, b, starts = _small_workload()
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[10], mixed=mixed,
                             fine_prec=fine if mixed else 2)
    h = wm.mg_setup(U, dims, 0.1, p, starts=starts)
    x = np.zeros_like(b)
    status, st = wm.mg_solve(h, b, x, 1e-10)
    assert status == wm.MG_OK
    assert st[0]["true_rel_residual"] <= 1e-10
    assert _true_rel(U, 0.1, x, b) <= 1e-10
    xl = scipy.linalg.lu_solve(lu_small, b.reshape(-1)).reshape(b.shape)
    assert rel_err(x, xl) < 1e-8
    if mixed:
        assert st[0]["fine_dslash_f64"] <= st[0]["reliable_updates"] + 1


def test_plain_gpu_iterations_match_oracle():
    """Plain FP64: same hierarchy and same arithmetic, so the outer iteration count equals the oracle's."""
    wm = require_gpu()
    dims, U, b, starts = _small_workload()
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[10])
    h = wm.mg_setup(U, dims, 0.1, p, starts=starts)
    x = np.zeros_like(b)
    _, st = wm.mg_solve(h, b, x, 1e-10)
    hier = mg.mg_setup(U, 0.1, [dict(block=(2, 2, 2, 2), nv=8, sweeps=10)],
                       [list(starts[0].reshape((8,) + lattice(dims) + (12,)))])
    xo, info = mg.mg_solve(hier, b.reshape(lattice(dims) + (12,)), tol=1e-10)
    assert abs(st[0]["iters"] - info["iters"]) <= 1
    assert rel_err(x.reshape(xo.shape), xo) < 1e-9


def test_unpreconditioned_gcr(lu_small):
    wm = require_gpu()
    dims, U, b, _ = _small_workload()
    p = wm.mg_default_params(n_levels=1)
    h = wm.mg_setup(U, dims, 0.1, p)
    x = np.zeros_like(b)
    _, st = wm.mg_solve(h, b, x, 1e-10)
    assert _true_rel(U, 0.1, x, b) <= 1e-10
    xl = scipy.linalg.lu_solve(lu_small, b.reshape(-1)).reshape(b.shape)
    assert rel_err(x, xl) < 1e-8


@pytest.mark.parametrize("mixed,extra", [(0, {}), (1, {}), (1, dict(coarse_mma=1)), (1, dict(coarse_prec=2)),
                                         (1, dict(coarsest_f64=1)),
                                         (1, dict(fine_prec=3, coarse_prec=3))])
def test_three_level_solve_and_multi_rhs(mixed, extra):
    """Five right-hand sides (the coarsest inverse is applied as one tiled product), every
    storage scheme of the coarse levels: FP64, FP32 (CUDA cores / BF16 tensor cores), FP16, BF16."""
    wm = require_gpu()
    dims = (8, 8, 8, 8)
    mass = -0.2
    U = inputs.random_gauge(dims, 4)
    nrhs = 5
    b = np.stack([inputs.gaussian_spinor(dims, 20 + r) for r in range(nrhs)])
    b[1] = inputs.point_source(dims, 2, 1)
    p = wm.mg_default_params(n_levels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 6], setup_sweeps=[8, 8],
                             mixed=mixed, **extra)
    h = wm.mg_setup(U, dims, mass, p)
    x = np.zeros_like(b)
    _, st = wm.mg_solve(h, b, x, 1e-10)
    for r in range(nrhs):
        assert _true_rel(U, mass, x[r], b[r]) <= 1e-10, r
        assert st[r]["true_rel_residual"] <= 1e-10
    # the batched solve and a solve of one rhs alone give the same x
    x1 = np.zeros_like(b[1])
    wm.mg_solve(h, np.ascontiguousarray(b[1]), x1, 1e-10)
    assert rel_err(x1, x[1]) < 1e-8


def test_device_buffers_and_initial_guess():
    wm = require_gpu()
    dims, U, b, starts = _small_workload()
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[10], mixed=1)
    h = wm.mg_setup(torch.from_numpy(U).cuda(), dims, 0.1, p, starts=starts)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    wm.mg_solve(h, bd, xd, 1e-10)
    assert _true_rel(U, 0.1, xd.cpu().numpy(), b) <= 1e-10
    # starting from the solution needs no iteration
    _, st = wm.mg_solve(h, bd, xd, 1e-10)
    assert st[0]["iters"] == 0


def test_iteration_cap_reports_no_convergence():
    wm = require_gpu()
    dims, U, b, _ = _small_workload()
    p = wm.mg_default_params(n_levels=1, max_iter=3)
    h = wm.mg_setup(U, dims, 0.1, p)
    x = np.zeros_like(b)
    status, st = wm.mg_solve(h, b, x, 1e-10, raise_on_noconv=False)
    assert status == wm.MG_ENOCONV
    assert st[0]["iters"] == 3
    assert abs(st[0]["true_rel_residual"] - _true_rel(U, 0.1, x, b)) < 1e-12


def test_bad_arguments():
    wm = require_gpu()
    dims, U, b, _ = _small_workload()
    p = wm.mg_default_params(n_levels=2, block=[(3, 2, 2, 2)], nv=[8])
    with pytest.raises(wm.MgError) as e:
        wm.mg_setup(U, dims, 0.1, p)
    assert e.value.status == wm.MG_EINVAL
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[97])
    with pytest.raises(wm.MgError):
        wm.mg_setup(U, dims, 0.1, p)


@pytest.mark.parametrize("mixed", [0, 1])
def test_graph_replay_equals_eager_launches(mixed):
    """The V-cycle captured as a CUDA graph gives bit-identical iterates to eager launches."""
    wm = require_gpu()
    dims, U, b, starts = _small_workload()
    xs, its = [], []
    for graphs in (1, 0):
        p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[10], mixed=mixed,
                                 use_graphs=graphs)
        h = wm.mg_setup(U, dims, 0.1, p, starts=starts)
        x = np.zeros_like(b)
        _, st = wm.mg_solve(h, b, x, 1e-10)
        xs.append(x)
        its.append(st[0]["iters"])
    assert its[0] == its[1]
    assert np.array_equal(xs[0], xs[1])


@pytest.mark.parametrize("mixed", [0, 1])
def test_four_level_solve(mixed):
    """The deepest hierarchy the library builds (8^4 -> 4^4 -> 2^4 -> 1^4, K-cycles on levels 1 and 2,
    exact solve on the one-site coarsest level): the true FP64 residual reaches 1e-10."""
    wm = require_gpu()
    dims = (8, 8, 8, 8)
    mass = -0.2
    U = inputs.random_gauge(dims, 8)
    b = np.stack([inputs.gaussian_spinor(dims, 60 + r) for r in range(3)])
    p = wm.mg_default_params(n_levels=4, block=[(2, 2, 2, 2)] * 3, nv=[8, 8, 6], setup_sweeps=[8, 8, 8],
                             mixed=mixed, coarse_mma=mixed)
    h = wm.mg_setup(U, dims, mass, p)
    x = np.zeros_like(b)
    _, st = wm.mg_solve(h, b, x, 1e-10)
    for r in range(3):
        assert _true_rel(U, mass, x[r], b[r]) <= 1e-10, r


def test_mixed_coarsest_solve_in_fp64():
    """coarsest_f64 = 1: the mixed hierarchy's coarsest solve is A^-1 r with an FP64 inverse; the
    solve reaches the tolerance with the iteration count of the FP32-inverse form within 2."""
    wm = require_gpu()
    dims = (4, 4, 4, 4)
    mass = 0.1
    U = inputs.random_gauge(dims, 0)
    b = inputs.gaussian_spinor(dims, 1)
    its = {}
    for f64 in (0, 1):
        p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[8], setup_sweeps=[10], mixed=1,
                                 coarsest_f64=f64)
        h = wm.mg_setup(U, dims, mass, p)
        x = np.zeros_like(b)
        _, st = wm.mg_solve(h, b, x, 1e-10)
        assert _true_rel(U, mass, x, b) <= 1e-10
        its[f64] = st[0]["iters"]
    assert abs(its[1] - its[0]) <= 2, its


@pytest.mark.parametrize("mixed", [0, 1])
def test_release_work_keeps_the_hierarchy(mixed):
    """mg_release_work hands the solve buffers back (the handle shrinks to its hierarchy) and the next
    solve, which takes fresh buffers and recaptures its cycle, returns the same x; a mass-per-RHS solve
    after it rebuilds its inverses."""
    wm = require_gpu()
    dims = (8, 4, 4, 8)
    U = inputs.random_gauge(dims, 5)
    p = wm.mg_default_params(n_levels=3, block=[(2, 2, 2, 2), (2, 2, 1, 2)], nv=[8, 6], setup_sweeps=[20, 20],
                             mixed=mixed)
    h = wm.mg_setup(U, dims, 0.1, p)
    b = np.stack([inputs.gaussian_spinor(dims, 20 + r) for r in range(3)])
    x1 = np.zeros_like(b)
    wm.mg_solve(h, b, x1, 1e-10)
    big = wm.mg_handle_bytes(h)
    freed = wm.mg_release_work(h)
    assert freed > 0 and wm.mg_handle_bytes(h) == big - freed
    x2 = np.zeros_like(b)
    wm.mg_solve(h, b, x2, 1e-10)
    assert rel_err(x2, x1) <= 1e-12
    masses = [0.1, 0.15, 0.2]
    xm = np.zeros_like(b)
    wm.mg_solve_masses(h, masses, b, xm, 1e-10)
    wm.mg_release_work(h)
    xm2 = np.zeros_like(b)
    wm.mg_solve_masses(h, masses, b, xm2, 1e-10)
    assert rel_err(xm2, xm) <= 1e-12
    for r, m in enumerate(masses):
        assert _true_rel(U, m, xm2[r], b[r]) <= 1e-10
