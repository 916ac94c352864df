"""GPU parity of the even-odd (Schur-complement) pieces against the oracle.

* eo_split / eo_merge move bits: the halves equal the oracle's parity split
  of the field as stored, exactly, and merge(split(x)) == x bit for bit;
* dslash_eo_apply and schur_apply against the oracle's H_eo, H_oe and S on
  the inputs as stored (tolerances as the full stencil's: FP64 1e-13, FP32
  2e-6, FP16 4e-3, BF16 3e-2 relative);
* the even-odd Krylov baselines reach the tolerance on the full system (the
  oracle recomputes the residual), take the oracle's iteration count on the
  Schur system within rounding, and need fewer iterations than the full
  system's;
* MG with the even-odd fine smoother: one V-cycle equals the oracle's
  (plain FP64), the outer iteration count matches, and the mixed-precision
  form converges to the same solution;
* odd extents are refused.
"""
import numpy as np
import pytest

from gpu_util import lattice, rel_err, require_gpu, torch
from oracle import dirac, evenodd, krylov
from oracle import multigrid as mg
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-6, 2: 4e-3, 3: 3e-2}
DIMS = (4, 2, 6, 4)  # Lx, Ly, Lz, Lt: 192 sites, two x-rows per (y, z, t) parity pattern


def _handle(wm, dims, mass, prec, U):
    kw = dict(n_levels=1)
    if prec != 0:
        kw.update(mixed=1, fine_prec=prec)
    return wm.mg_setup(U, dims, mass, wm.mg_default_params(**kw))


def _as_np(t):
    """Internal-layout tensor (complex or (..., 2) 16-bit) -> complex128 numpy, same leading shape."""
    if t.is_complex():
        return t.cpu().numpy().astype(np.complex128)
    a = t.float().cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def _stored_full(wm, h, prec, psi):
    """The fields psi (nrhs, ...) in internal layout of precision prec, and their values as stored."""
    nrhs = psi.shape[0]
    ext = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    full = wm.internal_empty(h, 0, prec, nrhs)
    wm.mg_field_to_internal(h, 0, prec, ext, full, nrhs)
    back = torch.empty_like(ext)
    wm.mg_field_from_internal(h, 0, prec, full, back, nrhs)
    return full, back.cpu().numpy()


def _half_of(o):
    """Oracle half field (V/2, 4, 3) -> internal half (3, V/2, 4): component c at [c // 4, site, c % 4]."""
    return np.ascontiguousarray(np.moveaxis(o.reshape(o.shape[0], 3, 4), 1, 0))


def _split_dev(wm, h, prec, full, nrhs):
    e = wm.internal_empty(h, 0, prec, nrhs, half=True)
    o = wm.internal_empty(h, 0, prec, nrhs, half=True)
    wm.eo_split(h, prec, full, e, o, nrhs)
    return e, o


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_split_and_merge_move_bits(prec):
    wm = require_gpu()
    U = inputs.random_gauge(DIMS, 1)
    h = _handle(wm, DIMS, 0.1, prec, U)
    nrhs = 2
    psi = np.stack([inputs.gaussian_spinor(DIMS, 20 + r) for r in range(nrhs)])
    full, stored = _stored_full(wm, h, prec, psi)
    e, o = _split_dev(wm, h, prec, full, nrhs)
    ge, go = _as_np(e), _as_np(o)
    for r in range(nrhs):
        we, wo = evenodd.split(stored[r])
        assert np.array_equal(ge[r], _half_of(we))
        assert np.array_equal(go[r], _half_of(wo))
    back = torch.zeros_like(full)
    wm.eo_merge(h, prec, e, o, back, nrhs)
    assert torch.equal(back, full)
    wm.eo_merge(h, prec, e, None, back, nrhs)
    for r in range(nrhs):
        be, bo = evenodd.split(np.moveaxis(_as_np(back)[r], 0, 1).reshape(lattice(DIMS) + (4, 3)))
        assert np.array_equal(be, evenodd.split(stored[r])[0]) and not np.any(bo)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("parity", [0, 1])
def test_dslash_eo_matches_oracle(prec, parity):
    wm = require_gpu()
    mass = -0.37
    U = inputs.random_gauge(DIMS, 3)
    h = _handle(wm, DIMS, mass, prec, U)
    nrhs = 3
    psi = np.stack([inputs.gaussian_spinor(DIMS, 30 + r) for r in range(nrhs)])
    full, stored = _stored_full(wm, h, prec, psi)
    e, o = _split_dev(wm, h, prec, full, nrhs)
    x, inp = (e, o) if parity == 0 else (o, e)
    out = wm.internal_empty(h, 0, prec, nrhs, half=True)
    a, b = 1.3, -0.45
    wm.dslash_eo_apply(h, prec, parity, x, inp, out, a, b, nrhs)
    got = _as_np(out)
    for r in range(nrhs):
        se, so = evenodd.split(stored[r])
        want = a * se + b * evenodd.hop_eo(U, so) if parity == 0 else a * so + b * evenodd.hop_oe(U, se)
        assert rel_err(got[r], _half_of(want)) < TOL[prec], (r, rel_err(got[r], _half_of(want)))
    # without the a-term
    wm.dslash_eo_apply(h, prec, parity, None, inp, out, 0.0, 1.0, nrhs)
    se, so = evenodd.split(stored[0])
    want = evenodd.hop_eo(U, so) if parity == 0 else evenodd.hop_oe(U, se)
    assert rel_err(_as_np(out)[0], _half_of(want)) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_schur_apply_matches_oracle(prec):
    wm = require_gpu()
    mass = -0.2
    dims = (4, 4, 4, 6)
    U = inputs.random_gauge(dims, 4)
    h = _handle(wm, dims, mass, prec, U)
    nrhs = 2
    psi = np.stack([inputs.gaussian_spinor(dims, 40 + r) for r in range(nrhs)])
    full, stored = _stored_full(wm, h, prec, psi)
    e, _ = _split_dev(wm, h, prec, full, nrhs)
    out = wm.internal_empty(h, 0, prec, nrhs, half=True)
    wm.schur_apply(h, prec, e, out, nrhs)
    got = _as_np(out)
    for r in range(nrhs):
        want = evenodd.schur(U, mass, evenodd.split(stored[r])[0])
        assert rel_err(got[r], _half_of(want)) < 2 * TOL[prec], rel_err(got[r], _half_of(want))


@pytest.mark.parametrize("method", ["bicgstab", "cgnr"])
def test_even_odd_krylov(method):
    wm = require_gpu()
    dims = (4, 4, 4, 8)
    mass = 0.05
    U = inputs.random_gauge(dims, 5)
    h = wm.mg_setup(U, dims, mass, wm.mg_default_params(n_levels=1))
    b = inputs.gaussian_spinor(dims, 6)
    tol = 1e-10
    full_m = wm.MG_KRYLOV_BICGSTAB if method == "bicgstab" else wm.MG_KRYLOV_CGNR
    eo_m = wm.MG_KRYLOV_BICGSTAB_EO if method == "bicgstab" else wm.MG_KRYLOV_CGNR_EO
    x = np.zeros_like(b)
    _, st = wm.krylov_solve(h, eo_m, b, x, tol)
    xf = np.zeros_like(b)
    _, stf = wm.krylov_solve(h, full_m, b, xf, tol)
    true = np.linalg.norm(b - dirac.wilson_dirac(U, x, mass)) / np.linalg.norm(b)
    assert st[0]["true_rel_residual"] <= tol and true <= 1.05 * tol, (st[0], true)
    assert rel_err(x, xf) < 1e-7
    assert st[0]["iters"] < stf[0]["iters"], (st[0]["iters"], stf[0]["iters"])
    # the oracle's method on the same Schur system, stopped at tol ||b||
    bh = evenodd.schur_rhs(U, mass, b)
    t2 = tol * np.linalg.norm(b) / np.linalg.norm(bh)

    def S(v):
        return evenodd.schur(U, mass, v)

    if method == "bicgstab":
        _, info = krylov.bicgstab(S, bh, t2)
    else:
        g5 = np.array([1.0, 1.0, -1.0, -1.0])[:, None]
        _, info = krylov.cgnr(S, lambda v: g5 * S(g5 * v), bh, t2)
    assert abs(st[0]["iters"] - info["iters"]) <= 2, (st[0]["iters"], info["iters"])


def _small(dims=(4, 4, 4, 4), nv=8):
    U = inputs.random_gauge(dims, 0)
    b = inputs.gaussian_spinor(dims, 1)
    starts = [np.stack(inputs.null_vector_starts(lattice(dims), 12, nv, 2)).reshape(nv, -1, 12)]
    return U, b, starts


def test_even_odd_smoother_cycle_and_solve():
    wm = require_gpu()
    dims = (4, 4, 4, 4)
    mass = 0.1
    U, b, starts = _small(dims)
    lat = lattice(dims)
    spec = dict(block=(2, 2, 2, 2), nv=8, sweeps=10)
    p = wm.mg_default_params(n_levels=2, block=[spec["block"]], nv=[8], setup_sweeps=[10], fine_smoother=1)
    h = wm.mg_setup(U, dims, mass, p, starts=starts)
    hier = mg.mg_setup(U, mass, [spec], [list(starts[0].reshape((8,) + lat + (12,)))], fine_smoother="eo")
    # one V-cycle
    rng = np.random.default_rng(5)
    r = rng.standard_normal(lat + (12,)) + 1j * rng.standard_normal(lat + (12,))
    rd = wm.internal_empty(h, 0, 0)
    wm.mg_field_to_internal(h, 0, 0, torch.from_numpy(r).cuda(), rd)
    ed = wm.internal_empty(h, 0, 0)
    wm.vcycle_apply(h, rd, ed)
    e = torch.empty((1,) + lat + (12,), dtype=torch.complex128, device="cuda")
    wm.mg_field_from_internal(h, 0, 0, ed, e)
    want = mg.vcycle(hier, 0, r, 2, 2, 0.8, (4,))
    assert rel_err(e.cpu().numpy().reshape(want.shape), want) < 1e-9
    # the outer solve
    x = np.zeros_like(b)
    _, st = wm.mg_solve(h, b, x, 1e-10)
    xo, info = mg.mg_solve(hier, b.reshape(lat + (12,)), tol=1e-10)
    assert abs(st[0]["iters"] - info["iters"]) <= 1, (st[0]["iters"], info["iters"])
    assert rel_err(x.reshape(xo.shape), xo) < 1e-9
    # MR smoother for comparison: the even-odd one needs no more outer iterations here
    p0 = wm.mg_default_params(n_levels=2, block=[spec["block"]], nv=[8], setup_sweeps=[10])
    h0 = wm.mg_setup(U, dims, mass, p0, starts=starts)
    x0 = np.zeros_like(b)
    _, st0 = wm.mg_solve(h0, b, x0, 1e-10)
    assert st[0]["iters"] <= st0[0]["iters"], (st[0]["iters"], st0[0]["iters"])


@pytest.mark.parametrize("fine", [2, 3])
def test_even_odd_smoother_mixed_multi_rhs(fine):
    wm = require_gpu()
    dims = (8, 8, 8, 8)
    mass = -0.25
    U = inputs.random_gauge(dims, 7)
    B = np.stack([inputs.gaussian_spinor(dims, 50 + r) for r in range(4)])
    out = {}
    for sm in (0, 1):
        p = wm.mg_default_params(n_levels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[12, 12],
                                 setup_sweeps=[8, 8], mixed=1, fine_prec=fine, fine_smoother=sm, seed=4)
        h = wm.mg_setup(U, dims, mass, p)
        X = np.zeros_like(B)
        status, st = wm.mg_solve(h, B, X, 1e-10)
        assert status == wm.MG_OK
        for r in range(B.shape[0]):
            true = np.linalg.norm(B[r] - dirac.wilson_dirac(U, X[r], mass)) / np.linalg.norm(B[r])
            assert true <= 1.05e-10, (sm, r, true)
        out[sm] = (X, [s["iters"] for s in st])
    assert rel_err(out[1][0], out[0][0]) < 1e-7
    assert max(out[1][1]) <= max(out[0][1]) + 2, (out[1][1], out[0][1])


def test_odd_extents_are_refused():
    wm = require_gpu()
    dims = (4, 3, 4, 4)
    U = inputs.random_gauge(dims, 0)
    p = wm.mg_default_params(n_levels=2, block=[(2, 3, 2, 2)], nv=[4], setup_sweeps=[2], fine_smoother=1)
    with pytest.raises(wm.MgError) as e:
        wm.mg_setup(U, dims, 0.1, p)
    assert e.value.status == wm.MG_EINVAL
    h = wm.mg_setup(U, dims, 0.1, wm.mg_default_params(n_levels=1))
    b = inputs.gaussian_spinor(dims, 1)
    with pytest.raises(wm.MgError):
        wm.krylov_solve(h, wm.MG_KRYLOV_BICGSTAB_EO, b, np.zeros_like(b), 1e-8)
