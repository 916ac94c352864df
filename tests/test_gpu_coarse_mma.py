"""Tensor-core coarse stencil (BF16 mma.sync, FP32 accumulation) against the oracle stencil.

The Galerkin coarse operator of level 1 is applied to several right-hand
sides on tensor cores and compared with the oracle's stencil_apply of the
FP64 operator the library exports.  BF16 rounds both operands to 8
mantissa bits, so the tolerance is 2e-2 relative (a few units of 2^-8 on a
sum of 9 n terms); the CUDA-core FP32 path of the same handle meets 1e-5.
A full three-level solve with the tensor-core coarse level still reaches
the true FP64 residual.
"""
import numpy as np
import pytest

from gpu_util import rel_err, require_gpu, torch
from oracle import dirac
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


def _handle(wm, nv0, mma, dims=(8, 8, 8, 8)):
    U = inputs.random_gauge(dims, 6)
    p = wm.mg_default_params(n_levels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[nv0, 4], setup_sweeps=[10, 10],
                             mixed=1, coarse_mma=mma)
    return wm.mg_setup(U, dims, -0.1, p), U


@pytest.mark.parametrize("nv0", [8, 10, 24])
@pytest.mark.parametrize("nrhs", [1, 5, 24])
def test_mma_coarse_apply_matches_oracle(nv0, nrhs):
    wm = require_gpu()
    h, _ = _handle(wm, nv0, 1)
    dims, nc, _ = wm.mg_level_info(h, 1)
    shape = (nrhs, dims[3], dims[2], dims[1], dims[0], nc)
    rng = np.random.default_rng(nv0 + nrhs)
    y = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    yi = wm.internal_empty(h, 1, wm.MG_F32, nrhs)
    wm.mg_field_to_internal(h, 1, wm.MG_F32, torch.from_numpy(y).cuda(), yi, nrhs)
    oi = wm.internal_empty(h, 1, wm.MG_F32, nrhs)
    wm.coarse_apply(h, 1, wm.MG_F32, yi, oi, nrhs)
    out = torch.empty(shape, dtype=torch.complex128, device="cuda")
    wm.mg_field_from_internal(h, 1, wm.MG_F32, oi, out, nrhs)
    out = out.cpu().numpy()
    A = wm.mg_get_coarse_op(h, 1).reshape((9,) + shape[1:5] + (nc, nc))
    for r in range(nrhs):
        assert rel_err(out[r], dirac.stencil_apply(A, y[r])) < 2e-2, r


def test_mma_three_level_multi_rhs_solve():
    wm = require_gpu()
    h, U = _handle(wm, 8, 1)
    b = np.stack([inputs.gaussian_spinor((8, 8, 8, 8), 40 + r) for r in range(6)])
    x = np.zeros_like(b)
    _, st = wm.mg_solve(h, b, x, 1e-10)
    for r in range(6):
        assert np.linalg.norm(b[r] - dirac.wilson_dirac(U, x[r], -0.1)) <= 1e-10 * np.linalg.norm(b[r])
