"""GPU BiCGstab and CG-on-the-normal-equations baselines (Secs. 4-5) against the oracle.

Same FP64 arithmetic on both sides in the same order of operations up to
the reduction order, so the iteration counts agree to within one and the
solutions agree with dense LU to the conditioning of the solve.
"""
import numpy as np
import pytest
import scipy.linalg

from gpu_util import lattice, require_gpu, torch
from oracle import dirac
from oracle import krylov
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,mass", [((4, 4, 4, 4), 0.1), ((6, 4, 2, 4), -0.3)])
def test_krylov_baselines_match_oracle(dims, mass):
    wm = require_gpu()
    U = inputs.random_gauge(dims, 2)
    lat = lattice(dims)
    shp = lat + (4, 3)
    b = inputs.gaussian_spinor(dims, 3)
    p = wm.mg_default_params(n_levels=1)
    h = wm.mg_setup(U, dims, mass, p)

    def A(v):
        return dirac.wilson_dirac(U, v.reshape(shp), mass).reshape(v.shape)

    def Ad(v):
        return dirac.apply_gamma5(dirac.wilson_dirac(U, dirac.apply_gamma5(v.reshape(shp)), mass)).reshape(v.shape)

    D = dirac.dense_matrix(A, (b.size,))
    xl = scipy.linalg.solve(D, b.reshape(-1))
    for method in (wm.MG_KRYLOV_BICGSTAB, wm.MG_KRYLOV_CGNR):
        x = np.zeros_like(b)
        _, st = wm.krylov_solve(h, method, b, x, 1e-10)
        r = b.reshape(-1) - D @ x.reshape(-1)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b) * 1.001
        assert np.linalg.norm(x.reshape(-1) - xl) < 1e-8 * np.linalg.norm(xl)
        if method == wm.MG_KRYLOV_BICGSTAB:
            _, info = krylov.bicgstab(A, b.reshape(-1), tol=1e-10)
        else:
            _, info = krylov.cgnr(A, Ad, b.reshape(-1), tol=1e-10)
        assert abs(st[0]["iters"] - info["iters"]) <= 1, (method, st[0]["iters"], info["iters"])
        assert st[0]["true_rel_residual"] <= 1e-10


def test_krylov_device_buffers_and_cap():
    wm = require_gpu()
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 1)
    h = wm.mg_setup(U, dims, 0.1, wm.mg_default_params(n_levels=1))
    b = torch.from_numpy(np.stack([inputs.gaussian_spinor(dims, 5 + r) for r in range(2)])).cuda()
    x = torch.zeros_like(b)
    _, st = wm.krylov_solve(h, wm.MG_KRYLOV_BICGSTAB, b, x, 1e-10)
    assert all(s["true_rel_residual"] <= 1e-10 for s in st)
    x.zero_()
    status, st = wm.krylov_solve(h, wm.MG_KRYLOV_CGNR, b, x, 1e-10, max_iter=3, raise_on_noconv=False)
    assert status == wm.MG_ENOCONV and st[0]["iters"] == 3 and st[0]["true_rel_residual"] > 1e-10
