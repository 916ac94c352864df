"""Tensor-core restriction / prolongation for several right-hand sides (Sec. 3, Eq. 3.2).

The library's own P (exported in FP64) defines the expected values, computed
with the oracle's restrict / prolong; the vectors enter in 16-bit storage.
Tolerances: against the FP64 oracle, the 16-bit rounding of the inputs
(2^-11 relative for FP16, 2^-8 for BF16, times a few for the sums); against
the one-right-hand-side CUDA-core kernels (same 16-bit inputs, FP32
arithmetic, other summation order) 1e-5 for the restriction, and for the
prolongation the FP16/BF16 rounding of the coarse FP32 input that the
tensor-core path adds.
"""
import numpy as np
import pytest

from gpu_util import lattice, rel_err, require_gpu, torch
from oracle import multigrid as mg
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle_P(vecs, nv, nhalf):
    """Library prolongator vectors (nv, lattice..., ncomp) -> oracle P (lattice..., ncomp, 2 nv)."""
    v = np.moveaxis(vecs, 0, -1)  # lattice + (ncomp, nv)
    P = np.zeros(v.shape[:-1] + (2 * nv,), dtype=np.complex128)
    P[..., :nhalf, :nv] = v[..., :nhalf, :]
    P[..., nhalf:, nv:] = v[..., nhalf:, :]
    return P


def _to_dev(wm, h, level, arr, prec, nrhs):
    t = wm.internal_empty(h, level, prec, nrhs)
    wm.mg_field_to_internal(h, level, prec, torch.from_numpy(np.ascontiguousarray(arr)).cuda(), t, nrhs)
    return t


def _to_host(wm, h, level, t, shape, prec, nrhs):
    e = torch.empty(shape, dtype=torch.complex128, device="cuda")
    wm.mg_field_from_internal(h, level, prec, t, e, nrhs)
    return e.cpu().numpy()


CASES = [
    ((4, 4, 4, 4), (2, 2, 2, 2), 8, 5, 2),      # one K chunk (len 96), one M tile
    ((8, 8, 8, 8), (4, 4, 4, 4), 20, 24, 2),    # 12 K chunks (len 1536), two M tiles, 3 rhs tiles
    ((8, 4, 4, 8), (4, 2, 2, 4), 24, 64, 3),    # BF16, 64 right-hand sides (8 rhs tiles)
    ((4, 4, 4, 4), (2, 2, 2, 2), 40, 3, 2),     # nv = 40: three M tiles, the CUDA-core kernels
]


@pytest.mark.parametrize("dims,block,nv,nrhs,prec", CASES)
def test_multi_rhs_transfers(dims, block, nv, nrhs, prec):
    wm = require_gpu()
    U = inputs.random_gauge(dims, 1)
    p = wm.mg_default_params(n_levels=2, block=[block], nv=[nv], setup_sweeps=[3], mixed=1, fine_prec=prec)
    h = wm.mg_setup(U, dims, 0.1, p)
    lat = lattice(dims)
    vecs = wm.mg_get_prolongator(h, 0).reshape((nv,) + lat + (12,))
    blk = mg.Blocking(lat, block, 12)
    P = _oracle_P(vecs, nv, 6)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((nrhs,) + lat + (12,)) + 1j * rng.standard_normal((nrhs,) + lat + (12,))
    xc = rng.standard_normal((nrhs,) + blk.coarse + (2 * nv,)) + 1j * rng.standard_normal((nrhs,) + blk.coarse + (2 * nv,))
    eps = 2.0 ** -11 if prec == 2 else 2.0 ** -8
    # restriction: 16-bit in, FP32 out
    rd = _to_dev(wm, h, 0, r, prec, nrhs)
    out = wm.internal_empty(h, 1, 1, nrhs)
    wm.restrict_apply(h, 0, prec, rd, out, nrhs)
    got = _to_host(wm, h, 1, out, xc.shape, 1, nrhs)
    want = np.stack([mg.restrict(P, blk, r[i]) for i in range(nrhs)])
    assert rel_err(got, want) < 8 * eps, rel_err(got, want)
    for i in (0, nrhs - 1):  # the one-rhs kernel on the same 16-bit input
        out1 = wm.internal_empty(h, 1, 1, 1)
        wm.restrict_apply(h, 0, prec, rd[i:i + 1].contiguous(), out1, 1)
        assert rel_err(_to_host(wm, h, 1, out1, xc.shape[1:], 1, 1), got[i]) < 1e-5
    # prolongation: FP32 in, 16-bit out
    cd = _to_dev(wm, h, 1, xc, 1, nrhs)
    fo = wm.internal_empty(h, 0, prec, nrhs)
    wm.prolong_apply(h, 0, prec, cd, fo, nrhs)
    got = _to_host(wm, h, 0, fo, r.shape, prec, nrhs)
    want = np.stack([mg.prolong(P, blk, xc[i]) for i in range(nrhs)])
    assert rel_err(got, want) < 8 * eps, rel_err(got, want)
    for i in (0, nrhs - 1):
        fo1 = wm.internal_empty(h, 0, prec, 1)
        wm.prolong_apply(h, 0, prec, cd[i:i + 1].contiguous(), fo1, 1)
        assert rel_err(_to_host(wm, h, 0, fo1, r.shape[1:], prec, 1), got[i]) < 4 * eps
