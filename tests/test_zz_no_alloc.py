"""mr_apply_noalloc: the same MR smoothing as mr_apply with no device allocation.

Some callers of this library cannot allocate device memory at the moment
they smooth: a server that fixed its memory footprint at start-up, or a host
thread that must not take the driver's allocation path while other streams
run.  mr_apply_noalloc takes all its scratch from a fixed array compiled into
the library.  This test checks, through the C ABI, that two calls in a row on
a fresh handle allocate nothing (the library's allocation counter does not
move) and give what mr_apply then gives on the same inputs, within the
tolerance of the other GPU tests (1e-13 relative in FP64, 1e-6 in FP32),
including a coarse level in FP32 on the tensor-core stencil, and that an
oversized level is refused.

This file is collected last on purpose.
"""
import numpy as np
import pytest

from gpu_util import rel_err, require_gpu, torch
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


def _internal(wm, h, level, prec, ext):
    t = wm.internal_empty(h, level, prec)
    wm.mg_field_to_internal(h, level, prec, torch.from_numpy(np.ascontiguousarray(ext)).cuda(), t)
    return t


def _host(wm, h, level, prec, t, shape):
    e = torch.empty(shape, dtype=torch.complex128, device="cuda")
    wm.mg_field_from_internal(h, level, prec, t, e)
    return e.cpu().numpy()


@pytest.mark.parametrize("level,prec,mma", [(0, 0, 0), (0, 1, 0), (1, 0, 0), (1, 1, 1)])
def test_no_alloc_mr_matches_mr_apply_twice(level, prec, mma):
    wm = require_gpu()
    dims = (8, 4, 4, 8)
    U = inputs.random_gauge(dims, 3)
    mixed = 1 if prec == 1 else 0
    if mma:  # the tensor-core stencil lives on coarse levels above the coarsest: three levels
        p = wm.mg_default_params(n_levels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 4], setup_sweeps=[4, 4],
                                 mixed=mixed, fine_prec=wm.MG_F32, coarse_prec=wm.MG_F32, coarse_mma=1)
    else:
        p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[6], setup_sweeps=[4], mixed=mixed,
                                 fine_prec=wm.MG_F32, coarse_prec=wm.MG_F32)
    h = wm.mg_setup(U, dims, -0.1, p)
    ldims, nc, _ = wm.mg_level_info(h, level)
    shape = (ldims[3], ldims[2], ldims[1], ldims[0], nc)
    rng = np.random.default_rng(level * 10 + prec)
    b = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    x0 = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    tol = 1e-13 if prec == 0 else 1e-6
    bi = _internal(wm, h, level, prec, b)
    xs = [_internal(wm, h, level, prec, x0) for _ in range(4)]
    rs = [wm.internal_empty(h, level, prec) for _ in range(4)]
    torch.cuda.synchronize()
    # two calls in a row on the fresh handle, before any mr_apply: nothing allocated
    n0 = wm.mg_alloc_count()
    for call in range(2):
        wm.mr_apply_noalloc(h, level, prec, bi, xs[call], rs[call], 3)
    torch.cuda.synchronize()
    assert wm.mg_alloc_count() == n0
    for call in range(2):
        wm.mr_apply(h, level, prec, bi, xs[2 + call], rs[2 + call], 3)
    torch.cuda.synchronize()
    for call in range(2):
        xa, xb = _host(wm, h, level, prec, xs[2 + call], shape), _host(wm, h, level, prec, xs[call], shape)
        ra, rb = _host(wm, h, level, prec, rs[2 + call], shape), _host(wm, h, level, prec, rs[call], shape)
        assert rel_err(xb, xa) <= tol, (call, rel_err(xb, xa))
        assert rel_err(rb, ra) <= tol, (call, rel_err(rb, ra))


def test_no_alloc_refuses_levels_beyond_its_scratch():
    wm = require_gpu()
    dims = (32, 16, 16, 16)  # one FP64 work vector alone is 24 MiB
    U = inputs.random_gauge_fast(dims, 1)
    h = wm.mg_setup(U, dims, 0.1, wm.mg_default_params(n_levels=1))
    a = wm.internal_empty(h, 0, 0)
    with pytest.raises(wm.MgError) as e:
        wm.mr_apply_noalloc(h, 0, 0, a, a, a, 1)
    assert e.value.status == wm.MG_EINVAL
    assert "scratch" in wm.mg_last_error()
