"""A mass per right-hand side in one solve equals the retargeted single-mass solves (to the solution's
tolerance; the per-right-hand-side shift enters the coarse stencils as an added term, not a rounded
diagonal, so not bit for bit)."""
import numpy as np
import pytest

from gpu_util import rel_err, require_gpu
from oracle import dirac
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mixed,levels", [(0, 2), (1, 2), (1, 3)])
def test_mass_per_rhs_equals_retargeted_solves(mixed, levels):
    wm = require_gpu()
    dims = (8, 8, 4, 8)
    U = inputs.random_gauge(dims, 9)
    blocks = [(2, 2, 2, 2)] + ([(2, 2, 1, 2)] if levels == 3 else [])
    p = wm.mg_default_params(n_levels=levels, block=blocks, nv=[8] * (levels - 1), setup_sweeps=[20] * (levels - 1),
                             mixed=mixed, coarse_mma=mixed)
    h0 = wm.mg_setup(U, dims, -0.1, p)
    masses = [0.2, 0.05, 0.0, 0.05, -0.05]
    B = np.stack([inputs.gaussian_spinor(dims, 30 + r) for r in range(len(masses))])
    X = np.zeros_like(B)
    status, st = wm.mg_solve_masses(h0, masses, B, X, 1e-10)
    assert status == wm.MG_OK
    for r, m in enumerate(masses):
        rel = np.linalg.norm(B[r] - dirac.wilson_dirac(U, X[r], m)) / np.linalg.norm(B[r])
        assert rel <= 1.05e-10 and st[r]["true_rel_residual"] <= 1e-10, (r, rel)
        h = wm.mg_retarget(h0, m)
        x = np.zeros_like(B[r])
        wm.mg_solve(h, B[r], x, 1e-10)
        assert rel_err(X[r], x) < 1e-8, (r, m)
    # afterwards the handle solves at its own mass again
    x = np.zeros_like(B[0])
    _, s0 = wm.mg_solve(h0, B[0], x, 1e-10)
    assert np.linalg.norm(B[0] - dirac.wilson_dirac(U, x, -0.1)) <= 1.05e-10 * np.linalg.norm(B[0])
