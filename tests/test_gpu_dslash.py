"""GPU parity of the level-0 Wilson-Dirac stencil (dslash_apply) against the oracle.

Tolerances: FP64 storage and arithmetic 1e-13 relative (the FP64 target);
FP32 2e-6; FP16 storage (FP32 arithmetic) 4e-3 and BF16 3e-2, i.e. a few
units of the storage rounding (2^-11, 2^-8) of inputs and links.
"""
import numpy as np
import pytest

from gpu_util import lattice, rel_err, require_gpu, torch
from oracle import dirac
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-6, 2: 4e-3, 3: 3e-2}


def _handle(wm, dims, mass, mixed_prec=None, U=None):
    U = inputs.random_gauge(dims, 3) if U is None else U
    kw = dict(n_levels=1)
    if mixed_prec is not None:
        kw.update(mixed=1, fine_prec=mixed_prec)
    p = wm.mg_default_params(**kw)
    return wm.mg_setup(U, dims, mass, p), U


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 2, 4), (6, 5, 4, 7), (2, 2, 2, 2), (1, 3, 1, 2)])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_dslash_matches_oracle(dims, prec):
    wm = require_gpu()
    mass = -0.37
    h, U = _handle(wm, dims, mass, None if prec == 0 else prec)
    nrhs = 3
    psi = np.stack([inputs.gaussian_spinor(dims, 10 + r) for r in range(nrhs)])
    ext = torch.from_numpy(psi).cuda()
    inp = wm.internal_empty(h, 0, prec, nrhs)
    out = wm.internal_empty(h, 0, prec, nrhs)
    wm.mg_field_to_internal(h, 0, prec, ext, inp, nrhs)
    wm.dslash_apply(h, prec, inp, out, nrhs)
    got = torch.empty_like(ext)
    wm.mg_field_from_internal(h, 0, prec, out, got, nrhs)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    for r in range(nrhs):
        # compare with the oracle applied to the input as stored (rounded to prec)
        back = torch.empty_like(ext)
        wm.mg_field_from_internal(h, 0, prec, inp, back, nrhs)
        psi_s = back.cpu().numpy()[r]
        expect = dirac.wilson_dirac(U, psi_s, mass)
        assert rel_err(got[r], expect) < TOL[prec], (r, rel_err(got[r], expect))


def test_dslash_full_size_sampled_sites_and_gamma5():
    """32^3 x 64 (the large workload), FP16 and FP32 storage: sampled sites vs the
    per-site oracle, and gamma5-Hermiticity <y, g5 D x> = conj <x, g5 D y> on the whole lattice."""
    wm = require_gpu()
    dims = (32, 32, 32, 64)
    mass = -0.79
    U = inputs.random_gauge_fast(dims, 5)
    rng = np.random.default_rng(0)
    sites = [(0, 0, 0, 0), (31, 31, 31, 63), (5, 17, 0, 33)] + [
        tuple(int(rng.integers(0, L)) for L in dims) for _ in range(5)]
    for prec in (1, 2):
        h, _ = _handle(wm, dims, mass, prec, U=U)
        x = torch.from_numpy(inputs.gaussian_spinor(dims, 1)).cuda()
        y = torch.from_numpy(inputs.gaussian_spinor(dims, 2)).cuda()
        xi, yi = wm.internal_empty(h, 0, prec), wm.internal_empty(h, 0, prec)
        Dx, Dy = wm.internal_empty(h, 0, prec), wm.internal_empty(h, 0, prec)
        wm.mg_field_to_internal(h, 0, prec, x, xi)
        wm.mg_field_to_internal(h, 0, prec, y, yi)
        wm.dslash_apply(h, prec, xi, Dx)
        wm.dslash_apply(h, prec, yi, Dy)
        ext = torch.empty_like(x)
        wm.mg_field_from_internal(h, 0, prec, Dx, ext)
        xs = torch.empty_like(x)
        wm.mg_field_from_internal(h, 0, prec, xi, xs)
        Dx_h, xs_h = ext.cpu().numpy(), xs.cpu().numpy()
        for s in sites:
            xx, yy, zz, tt = s
            e = dirac.wilson_dirac_site(U, xs_h, mass, s)
            assert rel_err(Dx_h[tt, zz, yy, xx], e) < TOL[prec] * 3
        # gamma5-Hermiticity over the whole lattice
        ys = torch.empty_like(y)
        wm.mg_field_from_internal(h, 0, prec, yi, ys)
        extY = torch.empty_like(y)
        wm.mg_field_from_internal(h, 0, prec, Dy, extY)
        g5 = torch.tensor([1, 1, -1, -1], dtype=torch.float64, device="cuda").view(4, 1)
        a = torch.vdot(ys.flatten(), (g5 * ext).flatten())
        b = torch.vdot(xs.flatten(), (g5 * extY).flatten()).conj()
        assert abs(a - b) / abs(a) < TOL[prec] * 10
        del h


def test_dslash_fused_residual_and_reduction_deterministic():
    """mr_apply(steps=0) computes r = b - D x through the fused residual form; run twice bit-equal."""
    wm = require_gpu()
    dims = (6, 5, 4, 7)
    mass = 0.05
    h, U = _handle(wm, dims, mass)
    b = inputs.gaussian_spinor(dims, 1)
    x = inputs.gaussian_spinor(dims, 2)
    outs = []
    for _ in range(2):
        bi, xi, ri = (wm.internal_empty(h, 0, 0) for _ in range(3))
        wm.mg_field_to_internal(h, 0, 0, torch.from_numpy(b).cuda(), bi)
        wm.mg_field_to_internal(h, 0, 0, torch.from_numpy(x).cuda(), xi)
        wm.mr_apply(h, 0, 0, bi, xi, ri, 3)
        rext = torch.empty(b.shape, dtype=torch.complex128, device="cuda")
        wm.mg_field_from_internal(h, 0, 0, ri, rext)
        xext = torch.empty(b.shape, dtype=torch.complex128, device="cuda")
        wm.mg_field_from_internal(h, 0, 0, xi, xext)
        outs.append((xext.cpu().numpy(), rext.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    from oracle import multigrid as mg
    lat = lattice(dims)
    A = lambda v: dirac.wilson_dirac(U, v.reshape(lat + (4, 3)), mass).reshape(lat + (12,))
    xo, ro = mg.mr_relax(A, b.reshape(lat + (12,)), x.reshape(lat + (12,)), 3, 0.8)
    assert rel_err(outs[0][0].reshape(xo.shape), xo) < 1e-13
    assert rel_err(outs[0][1].reshape(ro.shape), ro) < 1e-12


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("mode", [4, 3])
def test_dslash_large_lattice_whole_field(prec, mode):
    """16x8x8x8 with 6 right-hand sides (49,152 site x right-hand sides, above the 32,768 up to
    which the warp-per-hop kernel runs), so the one-thread-per-site stencil runs: every element
    against the oracle applied to the input as stored.  Tuner mode 4 forces the first launch
    shape (128 threads, one right-hand side per thread), mode 3 the last (256 threads, two per
    thread, each link shared by both); FP64 has one shape."""
    wm = require_gpu()
    dims = (16, 8, 8, 8)
    mass = -0.37
    h, U = _handle(wm, dims, mass, None if prec == 0 else prec)
    nrhs = 6
    psi = np.stack([inputs.gaussian_spinor(dims, 40 + r) for r in range(nrhs)])
    ext = torch.from_numpy(psi).cuda()
    inp = wm.internal_empty(h, 0, prec, nrhs)
    out = wm.internal_empty(h, 0, prec, nrhs)
    wm.mg_field_to_internal(h, 0, prec, ext, inp, nrhs)
    old = wm.mg_tune(mode)
    try:
        wm.dslash_apply(h, prec, inp, out, nrhs)
        torch.cuda.synchronize()
    finally:
        wm.mg_tune(old)
    got = torch.empty_like(ext)
    wm.mg_field_from_internal(h, 0, prec, out, got, nrhs)
    back = torch.empty_like(ext)
    wm.mg_field_from_internal(h, 0, prec, inp, back, nrhs)
    got, back = got.cpu().numpy(), back.cpu().numpy()
    for r in range(nrhs):
        expect = dirac.wilson_dirac(U, back[r], mass)
        assert rel_err(got[r], expect) < TOL[prec], (r, rel_err(got[r], expect))


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_mr_large_lattice_fused_dots(prec):
    """mr_apply on 16^4 (65,536 sites: the one-thread-per-site stencil with its fused dot
    products <A r|r>, ||A r||^2 feeding each MR coefficient) against the oracle's MR on the
    input as stored, one step and three steps."""
    wm = require_gpu()
    dims = (16, 16, 16, 16)
    mass = 0.05
    h, U = _handle(wm, dims, mass, None if prec == 0 else prec)
    b = inputs.gaussian_spinor(dims, 3)
    x = inputs.gaussian_spinor(dims, 4)
    from oracle import multigrid as mg
    lat = lattice(dims)
    A = lambda v: dirac.wilson_dirac(U, v.reshape(lat + (4, 3)), mass).reshape(lat + (12,))
    tol = {0: 1e-12, 1: 1e-5, 2: 1e-2, 3: 6e-2}[prec]
    for steps in (1, 3):
        bi, xi, ri = (wm.internal_empty(h, 0, prec) for _ in range(3))
        wm.mg_field_to_internal(h, 0, prec, torch.from_numpy(b).cuda(), bi)
        wm.mg_field_to_internal(h, 0, prec, torch.from_numpy(x).cuda(), xi)
        bs, xs = torch.empty(b.shape, dtype=torch.complex128, device="cuda"), torch.empty(
            b.shape, dtype=torch.complex128, device="cuda")
        wm.mg_field_from_internal(h, 0, prec, bi, bs)
        wm.mg_field_from_internal(h, 0, prec, xi, xs)
        wm.mr_apply(h, 0, prec, bi, xi, ri, steps)
        xext = torch.empty(b.shape, dtype=torch.complex128, device="cuda")
        rext = torch.empty(b.shape, dtype=torch.complex128, device="cuda")
        wm.mg_field_from_internal(h, 0, prec, xi, xext)
        wm.mg_field_from_internal(h, 0, prec, ri, rext)
        xo, ro = mg.mr_relax(A, bs.cpu().numpy().reshape(lat + (12,)), xs.cpu().numpy().reshape(lat + (12,)),
                             steps, 0.8)
        assert rel_err(xext.cpu().numpy().reshape(xo.shape), xo) < tol, (steps, "x")
        assert rel_err(rext.cpu().numpy().reshape(ro.shape), ro) < tol, (steps, "r")
