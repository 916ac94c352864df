"""Pins of the oracle V-cycle's structure (Sec. 2, Sec. 3 Eq. 3.5, Sec. 5) by dense linear algebra.

The cycle is checked stage by stage against matrices built column by column
from the pinned pieces (the fine operator, the prolongator, MR), with the
coarse solves done by numpy's dense solver and every minimisation by lstsq:

* pre-smoothing happens before the restriction, the coarse problem is the
  exact Galerkin one, and alpha minimises the residual left after
  pre-smoothing (not the cycle's input residual);
* post-smoothing is MR from zero on the residual left after the coarse
  correction, and it lowers the residual;
* on three levels the coarse equation gets ``coarse_cycles`` steps of flexible
  minimal residual over directions made by the next level's cycle; one step is
  not four.

A cycle that drops or reorders a stage, forms alpha against the wrong
residual or runs the wrong number of coarse steps fails one of these.
"""
import numpy as np

from oracle import dirac
from oracle import multigrid as mg
from paper_0811_4331_gb300 import inputs


def _lat(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx)


def _dense_prolongator(lev):
    nc = lev_ncomp_coarse(lev)
    return dirac.dense_matrix(lambda xc: mg.prolong(lev.P, lev.blk, xc), lev.blk.coarse + (nc,))


def lev_ncomp_coarse(lev):
    return lev.P.shape[-1]


def _lstsq_alpha(p, r):
    return np.linalg.lstsq(p.reshape(-1, 1), r.reshape(-1), rcond=None)[0][0]


def _two_level(seed=0):
    dims = (4, 2, 2, 2)
    U = inputs.random_gauge(dims, seed)
    lat = _lat(dims)
    starts = [inputs.null_vector_starts(lat, 12, 4, 50 + seed)]
    h = mg.mg_setup(U, 0.05, [dict(block=(2, 2, 2, 2), nv=4, sweeps=3)], starts)
    D = dirac.dense_matrix(h[0].apply, lat + (12,))
    Pd = _dense_prolongator(h[0])
    rng = np.random.default_rng(7 + seed)
    r = rng.standard_normal(lat + (12,)) + 1j * rng.standard_normal(lat + (12,))
    return h, D, Pd, r


def test_pre_smoothing_precedes_an_exact_galerkin_correction():
    """nu_pre = 2, nu_post = 0, exact coarse solve: e = e_pre + alpha P A_c^-1 P^+ (r - A e_pre)
    with A_c = P^+ A P and alpha the least-squares minimiser of ||(r - A e_pre) - alpha A x_c||."""
    h, D, Pd, r = _two_level()
    e_pre, res_pre = mg.mr_relax(h[0].apply, r, None, 2)
    Ac = Pd.conj().T @ D @ Pd
    ec = np.linalg.solve(Ac, Pd.conj().T @ res_pre.reshape(-1))
    xc = Pd @ ec
    alpha = _lstsq_alpha(D @ xc, res_pre)
    expect = e_pre.reshape(-1) + alpha * xc
    e = mg.vcycle(h, 0, r, nu_pre=2, nu_post=0).reshape(-1)
    assert np.linalg.norm(e - expect) < 1e-10 * np.linalg.norm(expect)
    # the coarse residual after the correction is (1 - alpha) times the one before it
    rc_after = Pd.conj().T @ (r.reshape(-1) - D @ e)
    rc_before = Pd.conj().T @ res_pre.reshape(-1)
    assert np.linalg.norm(rc_after - (1 - alpha) * rc_before) < 1e-10 * np.linalg.norm(rc_before)
    # alpha is not 1 here (smoothing moved the residual off the coarse space), so the
    # alternatives below differ measurably from the cycle
    assert abs(alpha - 1) > 1e-3
    # smoothing after the restriction instead of before: restrict r itself
    ec_wrong = np.linalg.solve(Ac, Pd.conj().T @ r.reshape(-1))
    wrong = e_pre.reshape(-1) + _lstsq_alpha(D @ (Pd @ ec_wrong), res_pre) * (Pd @ ec_wrong)
    assert np.linalg.norm(e - wrong) > 1e-6 * np.linalg.norm(expect)
    # alpha formed against the cycle's input residual instead of the smoothed one
    wrong_a = e_pre.reshape(-1) + _lstsq_alpha(D @ xc, r) * xc
    assert np.linalg.norm(e - wrong_a) > 1e-6 * np.linalg.norm(expect)


def test_post_smoothing_is_mr_on_the_corrected_residual():
    """V(2, 2) = V(2, 0) + MR^2 from zero on r - A V(2, 0), and it lowers the residual."""
    h, D, Pd, r = _two_level(seed=1)
    e0 = mg.vcycle(h, 0, r, nu_pre=2, nu_post=0)
    res0 = r - h[0].apply(e0)
    de, _ = mg.mr_relax(h[0].apply, res0, None, 2)
    e2 = mg.vcycle(h, 0, r, nu_pre=2, nu_post=2)
    assert np.linalg.norm(e2 - (e0 + de)) < 1e-10 * np.linalg.norm(e2)
    n0 = np.linalg.norm(r.reshape(-1) - D @ e0.reshape(-1))
    n2 = np.linalg.norm(r.reshape(-1) - D @ e2.reshape(-1))
    assert n2 < n0 * (1 - 1e-6)
    assert np.linalg.norm(de) > 1e-3 * np.linalg.norm(e0)


def _three_level():
    dims = (4, 4, 2, 2)
    U = inputs.random_gauge(dims, 4)
    lat = _lat(dims)
    starts = [inputs.null_vector_starts(lat, 12, 4, 60),
              inputs.null_vector_starts((1, 1, 2, 2), 8, 3, 61)]
    h = mg.mg_setup(U, 0.05, [dict(block=(2, 2, 2, 2), nv=4, sweeps=3),
                             dict(block=(2, 2, 1, 1), nv=3, sweeps=3)], starts)
    return h, lat


def _flexible_min_res(A1, b, precond, steps):
    """Flexible minimal residual written from its definition: direction z_k =
    precond(r_{k-1}); x_k minimises ||b - A1 x|| over span(z_1..z_k) (lstsq)."""
    Z = []
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(steps):
        Z.append(precond(r))
        Zm = np.stack(Z, axis=1)
        c = np.linalg.lstsq(A1 @ Zm, b, rcond=None)[0]
        x = Zm @ c
        r = b - A1 @ x
    return x


def _dense_cycle(ops, Ps, l, v, nu, steps):
    """The cycle restated on dense matrices: MR pre-smoothing (nu steps from zero), the
    restricted residual solved exactly on the coarsest level or by ``steps`` flexible
    minimal-residual steps over directions made by the next level's cycle, alpha by
    lstsq against the smoothed residual (Eq. 3.5), MR post-smoothing."""
    A = ops[l]
    e, res = mg.mr_relax(lambda y: A @ y, v, None, nu)
    rc = Ps[l].conj().T @ res
    if l + 1 == len(ops) - 1:
        ec = np.linalg.solve(ops[l + 1], rc)
    else:
        ec = _flexible_min_res(ops[l + 1], rc, lambda w: _dense_cycle(ops, Ps, l + 1, w, nu, steps), steps)
    xc = Ps[l] @ ec
    alpha = _lstsq_alpha(A @ xc, res)
    e = e + alpha * xc
    res = res - alpha * (A @ xc)
    de, _ = mg.mr_relax(lambda y: A @ y, res, None, nu)
    return e + de


def test_three_level_cycle_takes_coarse_cycles_flexible_steps():
    """V(1, 1) on three levels: the level-1 equation gets ``coarse_cycles`` steps of flexible
    minimal residual whose directions are the level-1 cycle (itself V(1, 1) with the exact
    level-2 solve) applied to the current residual; 4 steps are not 1."""
    h, lat = _three_level()
    D0 = dirac.dense_matrix(h[0].apply, lat + (12,))
    P0 = _dense_prolongator(h[0])
    A1 = P0.conj().T @ D0 @ P0
    P1 = _dense_prolongator(h[1])
    A2 = P1.conj().T @ A1 @ P1
    # the Galerkin products agree with the oracle's stencils (sanity of the dense pieces)
    A1s = dirac.dense_matrix(h[1].apply, h[1].lattice + (h[1].ncomp,))
    assert np.max(np.abs(A1 - A1s)) < 1e-12 * np.max(np.abs(A1))
    ops, Ps = [D0, A1, A2], [P0, P1]
    rng = np.random.default_rng(11)
    r = rng.standard_normal(lat + (12,)) + 1j * rng.standard_normal(lat + (12,))
    got = {}
    for steps in (4, 1):
        expect = _dense_cycle(ops, Ps, 0, r.reshape(-1), 1, steps)
        e = mg.vcycle(h, 0, r, nu_pre=1, nu_post=1, coarse_cycles=(steps,)).reshape(-1)
        assert np.linalg.norm(e - expect) < 1e-9 * np.linalg.norm(expect), steps
        got[steps] = e
    assert np.linalg.norm(got[4] - got[1]) > 1e-6 * np.linalg.norm(got[4])
    # more coarse steps leave a smaller level-1 residual (minimal residual over a growing space)
    rc = P0.conj().T @ mg.mr_relax(h[0].apply, r, None, 1)[1].reshape(-1)
    cyc = lambda w: _dense_cycle(ops, Ps, 1, w, 1, 4)
    n = [np.linalg.norm(rc - A1 @ _flexible_min_res(A1, rc, cyc, k)) for k in (1, 2, 3, 4)]
    assert all(n[k + 1] < n[k] * (1 - 1e-9) for k in range(3)), n
