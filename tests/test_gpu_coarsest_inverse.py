"""The coarsest level's dense inverse (Sec. 4: the coarsest system is solved exactly).

The blocked Gauss-Jordan elimination (panels of 8, 4 or 2 columns inside
rank-64 blocks) is checked against numpy's LU inverse of the coarse operator,
which is assembled column by column from the oracle's 9-point stencil applied to the
GPU's own FP64 coarse stencil.  Both are inverses of the same matrix, so
they agree to the elimination's rounding: relative error at most a small
multiple of the unit roundoff of the storage precision times the
1-norm condition number.  The shapes cover N a multiple of 64 and not, and
each panel width of both precisions.  (FP64 beyond 3072 unknowns, where a
panel's rows no longer fit in registers, runs the single-step form, whose N
launches each sweep the whole matrix; no hierarchy here has such a level.)
"""
import numpy as np
import pytest

from gpu_util import lattice, rel_err, require_gpu
from oracle import dirac
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu

# (lattice, block, nv, mixed): N = coarse sites x 2 nv
CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4), 9, 0),  # N = 288, FP64: panels of 8, a ragged last block of 32
    ((8, 8, 8, 8), (4, 4, 4, 4), 9, 1),  # N = 288, FP32: panels of 8
    ((8, 8, 4, 8), (2, 2, 2, 2), 8, 0),  # N = 2048, FP64: panels of 2
    ((8, 8, 4, 8), (2, 2, 2, 2), 8, 1),  # N = 2048, FP32: panels of 4
    ((8, 8, 8, 8), (2, 2, 2, 2), 8, 1),  # N = 4096, FP32: panels of 2
]


@pytest.mark.parametrize("dims,block,nv,mixed", CASES)
def test_coarsest_inverse_matches_lu(dims, block, nv, mixed):
    wm = require_gpu()
    U = inputs.random_gauge(dims, 11)
    p = wm.mg_default_params(n_levels=2, block=[block], nv=[nv], setup_sweeps=[20], mixed=mixed)
    h = wm.mg_setup(U, dims, 0.05, p)
    X = wm.mg_get_coarsest_inverse(h)
    cdims, nc, _ = wm.mg_level_info(h, 1)
    shape = lattice(cdims) + (nc,)
    A = wm.mg_get_coarse_op(h, 1).reshape((9,) + shape[:4] + (nc, nc))
    D = dirac.dense_matrix(lambda y: dirac.stencil_apply(A, y), shape)
    Xr = np.linalg.inv(D)
    kappa = np.linalg.norm(D, 1) * np.linalg.norm(Xr, 1)
    u = 2.0 ** -53 if not mixed else 2.0 ** -24
    err = rel_err(X, Xr)
    assert X.shape == D.shape
    assert err <= 64 * u * kappa, (err, kappa)
    # and X is a right inverse to the same order (the product is the check a caller sees)
    N = D.shape[0]
    assert np.linalg.norm(D @ X - np.eye(N)) / np.sqrt(N) <= 64 * u * kappa
