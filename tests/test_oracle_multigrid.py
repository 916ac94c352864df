"""Pins of the oracle multigrid pieces against mathematics the paper fixes.

* MR: exact residual-decrease identity and the least-squares optimality of alpha.
* Block QR: equals numpy's Householder QR up to column phases (a library
  routine), P^+ P = 1, structural chirality zeros, P P^+ v_i = v_i (Eq. 2.3).
* Restriction / prolongation: adjoint pair and R P = 1.
* Coarse stencil: equals the brute-force dense P^+ D P, for coarse extents
  1, 2 and 3, and on the second coarsening; coarse gamma5-Hermiticity.
* Two-grid special case: with Nv = 6 |b| the prolongator is square unitary,
  the coarse solve is exact and one MG-preconditioned GCR step solves.
* GCR: matches dense LU, minimal-residual monotonicity.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import dirac
from oracle import multigrid as mg
from paper_0811_4331_gb300 import inputs


def _lat(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx)


def _fine_apply(U, m):
    lat = U.shape[1:5]
    return lambda y: dirac.wilson_dirac(U, y.reshape(lat + (4, 3)), m).reshape(lat + (12,))


def test_alpha_is_least_squares_minimiser():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    r = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    a = mg.minimal_residual_coefficient(p, r)
    ls = np.linalg.lstsq(p[:, None], r, rcond=None)[0][0]
    assert abs(a - ls) < 1e-14 * abs(ls)
    assert mg.minimal_residual_coefficient(np.zeros(3, complex), r[:3]) == 0.0


def test_mr_residual_identity_and_monotone():
    """||r'||^2 = ||r||^2 - omega (2 - omega) |<p|r>|^2 / ||p||^2 per step, r' = b - D x' recomputed."""
    dims = (4, 4, 2, 2)
    U = inputs.random_gauge(dims, 1)
    A = _fine_apply(U, 0.1)
    lat = _lat(dims)
    b = inputs.gaussian_spinor(dims, 2).reshape(lat + (12,))
    omega = 0.8
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(5):
        p = A(r)
        pr = np.vdot(p, r)
        pp = np.vdot(p, p).real
        x1, r1 = mg.mr_relax(A, b, x, 1, omega)
        true = b - A(x1)
        assert np.allclose(r1, true, atol=1e-12)
        expect = np.vdot(r, r).real - omega * (2 - omega) * abs(pr) ** 2 / pp
        assert abs(np.vdot(true, true).real - expect) < 1e-11 * expect
        assert np.vdot(true, true).real < np.vdot(r, r).real
        x, r = x1, true


def test_mgs2_matches_householder_qr():
    rng = np.random.default_rng(3)
    Vb = rng.standard_normal((40, 7)) + 1j * rng.standard_normal((40, 7))
    Q = mg.mgs2(Vb)
    Qh, R = np.linalg.qr(Vb)
    ph = np.diag(R) / np.abs(np.diag(R))
    assert np.max(np.abs(Q - Qh * ph)) < 1e-13
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(7))) < 1e-14
    with pytest.raises(ArithmeticError):
        Vb[:, 3] = Vb[:, 0] * (0.5 - 2j)
        mg.mgs2(Vb)


def _hierarchy_pieces(dims, block, nv, sweeps, seed=0, m=0.1):
    U = inputs.random_gauge(dims, seed)
    lat = _lat(dims)
    A = _fine_apply(U, m)
    starts = inputs.null_vector_starts(lat, 12, nv, 100 + seed)
    cands = mg.relax_null_vectors(A, starts, sweeps)
    blk = mg.Blocking(lat, block, 12)
    P = mg.block_orthonormalize(cands, blk)
    return U, A, cands, blk, P


def test_prolongator_properties():
    dims = (4, 4, 4, 4)
    nv = 6
    U, A, cands, blk, P = _hierarchy_pieces(dims, (2, 2, 2, 2), nv, 4)
    # structural chirality zeros: [gamma5, P] = 0
    assert np.all(P[..., :6, nv:] == 0) and np.all(P[..., 6:, :nv] == 0)
    # P^+ P = 1 on the coarse space
    G = blk.block_sum(np.einsum("...ci,...cj->...ij", np.conj(P), P))
    assert np.max(np.abs(G - np.eye(2 * nv))) < 1e-14
    # P V_c = V: every candidate lies in the range of P (Eq. 2.3)
    for v in cands:
        proj = mg.prolong(P, blk, mg.restrict(P, blk, v))
        assert np.max(np.abs(proj - v)) < 1e-13


def test_restrict_prolong_adjoint():
    dims = (4, 4, 2, 4)
    U, A, cands, blk, P = _hierarchy_pieces(dims, (2, 2, 2, 2), 5, 3, seed=4)
    rng = np.random.default_rng(1)
    r = rng.standard_normal(blk.lattice + (12,)) + 1j * rng.standard_normal(blk.lattice + (12,))
    xc = rng.standard_normal(blk.coarse + (10,)) + 1j * rng.standard_normal(blk.coarse + (10,))
    lhs = np.vdot(mg.prolong(P, blk, xc), r)
    rhs = np.vdot(xc, mg.restrict(P, blk, r))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    assert np.max(np.abs(mg.restrict(P, blk, mg.prolong(P, blk, xc)) - xc)) < 1e-13


def _dense_check(dims, block, nv, sweeps, seed):
    U, A, cands, blk, P = _hierarchy_pieces(dims, block, nv, sweeps, seed)
    lat = _lat(dims)
    Af = dirac.wilson_stencil(U, 0.1)
    Ac = mg.coarse_stencil(Af, P, blk)
    D = dirac.dense_matrix(A, lat + (12,))
    Pd = dirac.dense_matrix(lambda xc: mg.prolong(P, blk, xc), blk.coarse + (2 * nv,))
    brute = Pd.conj().T @ D @ Pd
    dense = mg.dense_from_stencil(Ac)
    assert np.max(np.abs(brute - dense)) < 1e-13 * np.max(np.abs(brute))
    return Ac, blk


@pytest.mark.parametrize("dims,block", [((4, 4, 4, 4), (2, 2, 2, 2)),   # coarse extent 2
                                        ((6, 2, 2, 2), (2, 2, 2, 2)),   # extents 3 and 1
                                        ((2, 2, 2, 2), (2, 2, 2, 2))])  # a single aggregate
def test_coarse_stencil_equals_brute_force(dims, block):
    _dense_check(dims, block, 4, 3, seed=2)


def test_coarse_gamma5_hermiticity():
    """Gamma5 = diag(+1_Nv, -1_Nv) per coarse site: Gamma5 A_c Gamma5 = A_c^+ (from [gamma5, P] = 0)."""
    Ac, blk = _dense_check((4, 4, 4, 4), (2, 2, 2, 2), 4, 3, seed=5)
    Dc = mg.dense_from_stencil(Ac)
    nc = 8
    g5 = np.tile(np.r_[np.ones(nc // 2), -np.ones(nc // 2)], Dc.shape[0] // nc)
    lhs = g5[:, None] * Dc * g5[None, :]
    assert np.max(np.abs(lhs - Dc.conj().T)) < 1e-13


def test_second_coarsening_equals_brute_force():
    dims = (4, 4, 4, 4)
    nv0, nv1 = 4, 3
    U = inputs.random_gauge(dims, 8)
    lat = _lat(dims)
    starts = [inputs.null_vector_starts(lat, 12, nv0, 21),
              inputs.null_vector_starts((2, 2, 2, 2), 2 * nv0, nv1, 22)]
    levels = [dict(block=(2, 2, 2, 2), nv=nv0, sweeps=3), dict(block=(2, 2, 1, 1), nv=nv1, sweeps=3)]
    h = mg.mg_setup(U, 0.1, levels, starts)
    A1 = mg.dense_from_stencil(h[1].stencil)
    Pd = dirac.dense_matrix(lambda xc: mg.prolong(h[1].P, h[1].blk, xc), h[2].lattice + (2 * nv1,))
    brute = Pd.conj().T @ A1 @ Pd
    assert np.max(np.abs(brute - mg.dense_from_stencil(h[2].stencil))) < 1e-13 * np.max(np.abs(brute))
    # the coarse level keeps chirality in its own split (first nv0 comps +, last nv0 -)
    assert np.all(h[1].P[..., :nv0, nv1:] == 0) and np.all(h[1].P[..., nv0:, :nv1] == 0)


def test_unitary_prolongator_solves_in_one_step():
    """Nv = 6 |b|: P is square unitary, the coarse solve is exact, GCR converges in one step."""
    dims = (2, 2, 2, 2)
    U = inputs.random_gauge(dims, 0)
    lat = _lat(dims)
    starts = [inputs.null_vector_starts(lat, 12, 96, 7)]
    h = mg.mg_setup(U, 0.1, [dict(block=(2, 2, 2, 2), nv=96, sweeps=0)], starts)
    b = inputs.gaussian_spinor(dims, 3).reshape(lat + (12,))
    x, info = mg.mg_solve(h, b, tol=1e-11)
    assert info["iters"] == 1
    assert info["true_rel_residual"] < 1e-12


def test_gcr_matches_lu_and_is_monotone():
    dims = (2, 2, 2, 2)
    U = inputs.random_gauge(dims, 1)
    lat = _lat(dims)
    A = _fine_apply(U, 0.05)
    b = inputs.gaussian_spinor(dims, 2).reshape(lat + (12,))
    x, info = mg.fgcr(A, b, None, tol=1e-12, restart=200)
    D = dirac.dense_matrix(A, lat + (12,))
    xl = scipy.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(x - xl) < 1e-10 * np.linalg.norm(xl)
    assert info["iters"] <= 192
    h = np.array(info["history"])
    assert np.all(np.diff(h) <= 1e-15)


def test_two_level_mg_solve_small_workload():
    """4^4, U = exp(0.3 i H), m = 0.1, 2^4 blocks, Nv = 8, 10 setup sweeps, tol 1e-10."""
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 0)
    lat = _lat(dims)
    starts = [inputs.null_vector_starts(lat, 12, 8, 2)]
    h = mg.mg_setup(U, 0.1, [dict(block=(2, 2, 2, 2), nv=8, sweeps=10)], starts)
    b = inputs.gaussian_spinor(dims, 1).reshape(lat + (12,))
    x, info = mg.mg_solve(h, b, tol=1e-10)
    assert info["true_rel_residual"] <= 1e-10
    D = dirac.dense_matrix(h[0].apply, lat + (12,))
    xl = scipy.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(x - xl) < 1e-8 * np.linalg.norm(xl)
    # preconditioning pays: fewer outer iterations than plain GCR
    _, plain = mg.fgcr(h[0].apply, b, None, tol=1e-10)
    assert info["iters"] < plain["iters"]


def test_three_level_mg_solve():
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 3)
    lat = _lat(dims)
    starts = [inputs.null_vector_starts(lat, 12, 6, 31),
              inputs.null_vector_starts((2, 2, 2, 2), 12, 4, 32)]
    h = mg.mg_setup(U, 0.1, [dict(block=(2, 2, 2, 2), nv=6, sweeps=6),
                             dict(block=(2, 2, 1, 1), nv=4, sweeps=6)], starts)
    b = inputs.gaussian_spinor(dims, 4).reshape(lat + (12,))
    x, info = mg.mg_solve(h, b, tol=1e-10)
    assert info["true_rel_residual"] <= 1e-10


def test_gcr_fixed_is_minimal_residual_krylov():
    """n steps of GCR with the identity preconditioner solve an n x n system (Krylov space exhausted);
    one step with the exact inverse as preconditioner solves at once."""
    rng = np.random.default_rng(2)
    n = 12
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = mg.gcr_fixed(lambda v: A @ v, b, lambda r: r.copy(), n)
    assert np.linalg.norm(A @ x - b) < 1e-10 * np.linalg.norm(b)
    x1 = mg.gcr_fixed(lambda v: A @ v, b, lambda r: np.linalg.solve(A, r), 1)
    assert np.linalg.norm(A @ x1 - b) < 1e-12 * np.linalg.norm(b)
    # residual after k steps is the minimum over the k-dimensional Krylov space
    for k in (2, 5):
        xk = mg.gcr_fixed(lambda v: A @ v, b, lambda r: r.copy(), k)
        K = np.stack([np.linalg.matrix_power(A, j) @ b for j in range(k)], axis=1)
        c = np.linalg.lstsq(A @ K, b, rcond=None)[0]
        assert abs(np.linalg.norm(A @ xk - b) - np.linalg.norm(A @ (K @ c) - b)) < 1e-9 * np.linalg.norm(b)


def test_cycle_annihilates_the_coarse_space_without_smoothing():
    """With no smoothing and an exact coarse solve, M A x = x for x = P y: the
    correction P A_c^-1 P^+ A P y = P y and alpha = 1 (Eq. 3.5), so the
    adaptive step x + M(-A x) returns 0 (a sign error returns 2 x)."""
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 6)
    lat = _lat(dims)
    starts = [inputs.null_vector_starts(lat, 12, 6, 10)]
    h = mg.mg_setup(U, 0.05, [dict(block=(2, 2, 2, 2), nv=6, sweeps=4)], starts)
    rng = np.random.default_rng(3)
    y = rng.standard_normal(h[1].lattice + (12,)) + 1j * rng.standard_normal(h[1].lattice + (12,))
    x = mg.prolong(h[0].P, h[0].blk, y)
    x1 = x + mg.vcycle(h, 0, -h[0].apply(x), nu_pre=0, nu_post=0)
    assert np.linalg.norm(x1) < 1e-10 * np.linalg.norm(x)


def test_adaptive_setup_keeps_the_invariants_and_helps():
    """Adaptive steps on both levels of a 3-level hierarchy (Sec. 2: V^k grown by
    prototypes from the current cycle on A x = 0): P^+ P = 1 and the chirality
    zeros on every level (Eq. 2.3); both coarse stencils equal the brute-force
    Galerkin products of the final P's; the first Nv - adapt_nv columns of each
    chirality are those of the relaxation-only P with that many vectors (the
    adaptive vectors are appended, Gram-Schmidt runs in order); MG-GCR needs no
    more iterations than with Nv relaxation vectors."""
    dims = (4, 4, 4, 4)
    U = inputs.heatbath_gauge(dims, 6.0, 30, 5)
    lat = _lat(dims)
    starts = [inputs.null_vector_starts(lat, 12, 6, 11),
              inputs.null_vector_starts((2, 2, 2, 2), 12, 4, 12)]
    spec = [dict(block=(2, 2, 2, 2), nv=6, sweeps=3), dict(block=(2, 2, 1, 1), nv=4, sweeps=3)]
    aspec = [dict(sp, adapt_nv=3, adapt_steps=2, adapt_cycles=4) for sp in spec]
    b = inputs.gaussian_spinor(dims, 1).reshape(lat + (12,))
    h0 = mg.mg_setup(U, -0.6, spec, starts)
    _, before = mg.mg_solve(h0, b, tol=1e-10)
    h = mg.mg_setup(U, -0.6, aspec, starts)
    for l in range(2):
        P, blk = h[l].P, h[l].blk
        nv = P.shape[-1] // 2
        G = blk.block_sum(np.einsum("...ci,...cj->...ij", np.conj(P), P))
        assert np.max(np.abs(G - np.eye(2 * nv))) < 1e-12
        assert np.all(P[..., :blk.half, nv:] == 0) and np.all(P[..., blk.half:, :nv] == 0)
        D = dirac.dense_matrix(h[l].apply, h[l].lattice + (h[l].ncomp,))
        Pm = dirac.dense_matrix(lambda y: mg.prolong(P, blk, y), h[l + 1].lattice + (2 * nv,))
        Dc = dirac.dense_matrix(h[l + 1].apply, h[l + 1].lattice + (2 * nv,))
        assert np.max(np.abs(Dc - Pm.conj().T @ D @ Pm)) < 1e-11 * np.max(np.abs(D))
    # the relaxation part of V^k on level 0 is the prefix of the final P
    hr = mg.mg_setup(U, -0.6, [dict(spec[0], nv=3)], [starts[0][:3]])
    assert np.max(np.abs(h[0].P[..., [0, 1, 2, 6, 7, 8]] - hr[0].P)) < 1e-12
    assert np.max(np.abs(h[0].P - h0[0].P)) > 1e-2  # the adaptive vectors changed the rest
    x, after = mg.mg_solve(h, b, tol=1e-10)
    assert after["true_rel_residual"] <= 1e-10
    assert after["iters"] <= before["iters"], (after["iters"], before["iters"])


def test_adaptive_prototype_is_a_minimal_residual_solve_of_the_null_equation():
    """The prototype of an adaptive step is the current solver (flexible GCR with the
    V-cycle, Sec. 5) applied to A x = 0 (Sec. 2): ||A x|| never grows with the
    iteration count, across the restart at 8 too (a sign error in the right-hand
    side -A x doubles x instead); and with an exact preconditioner (P square
    unitary, so the V-cycle is A^-1) one iteration returns x = 0."""
    dims = (4, 4, 4, 4)
    U = inputs.heatbath_gauge(dims, 6.0, 30, 5)
    lat = _lat(dims)
    h = mg.mg_setup(U, -0.6, [dict(block=(2, 2, 2, 2), nv=6, sweeps=3)],
                    [inputs.null_vector_starts(lat, 12, 6, 11)])
    x0 = inputs.null_vector_starts(lat, 12, 1, 40)[0]
    cyc = dict(nu_pre=2, nu_post=2, omega=0.8, coarse_cycles=(4,), coarse_solver="gcr")
    res = [np.sqrt(mg.norm2(h[0].apply(x0)))]
    for k in range(1, 11):
        res.append(np.sqrt(mg.norm2(h[0].apply(mg.adaptive_prototype(h, 0, x0, k, cyc)))))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res, res[1:])), res
    assert res[-1] < 0.5 * res[0]
    # exact preconditioner: 2^4 lattice, one 2^4 block, Nv = 6|b| = 96
    d2 = (2, 2, 2, 2)
    U2 = inputs.random_gauge(d2, 1)
    l2 = _lat(d2)
    h2 = mg.mg_setup(U2, 0.1, [dict(block=(2, 2, 2, 2), nv=96, sweeps=0)],
                     [inputs.null_vector_starts(l2, 12, 96, 3)])
    y0 = inputs.null_vector_starts(l2, 12, 1, 41)[0]
    y1 = mg.adaptive_prototype(h2, 0, y0, 1, dict(cyc, nu_pre=0, nu_post=0))
    assert np.sqrt(mg.norm2(y1)) < 1e-10 * np.sqrt(mg.norm2(y0))


def test_coarse_stencil_brute_force_on_random_shapes():
    """The stencil Galerkin product against dense P^+ D P over random lattice and block shapes (coarse
    extents 1, 2, 3 in any direction), numbers of vectors and fields."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @st.composite
    def shapes(draw):
        block = tuple(draw(st.sampled_from([1, 2])) for _ in range(4))
        coarse = tuple(draw(st.sampled_from([1, 2, 3])) for _ in range(4))
        dims = tuple(b * c for b, c in zip(block, coarse))
        hyp.assume(int(np.prod(dims)) <= 48 and int(np.prod(block)) >= 2)
        nv = draw(st.integers(1, min(4, 6 * int(np.prod(block)))))
        return dims, block, nv

    @hyp.settings(max_examples=6, deadline=None, derandomize=True)
    @hyp.given(shape=shapes(), seed=st.integers(0, 1000))
    def check(shape, seed):
        dims, block, nv = shape
        _dense_check(dims, block, nv, 2, seed)

    check()


def test_prolongator_invariants_on_random_shapes():
    """P^+ P = 1, the chirality zeros and P P^+ v = v for every candidate (Eq. 2.3), and R = P^+ the
    adjoint of P, over random lattice and block shapes, vector counts and fields."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @st.composite
    def shapes(draw):
        block = tuple(draw(st.sampled_from([1, 2])) for _ in range(4))
        coarse = tuple(draw(st.sampled_from([1, 2])) for _ in range(4))
        hyp.assume(int(np.prod(block)) >= 2)
        nv = draw(st.integers(1, min(6, 6 * int(np.prod(block)))))
        return tuple(b * c for b, c in zip(block, coarse)), block, nv

    @hyp.settings(max_examples=8, deadline=None, derandomize=True)
    @hyp.given(shape=shapes(), seed=st.integers(0, 1000))
    def check(shape, seed):
        dims, block, nv = shape
        U, A, cands, blk, P = _hierarchy_pieces(dims, block, nv, 2, seed)
        assert np.all(P[..., :6, nv:] == 0) and np.all(P[..., 6:, :nv] == 0)
        G = blk.block_sum(np.einsum("...ci,...cj->...ij", np.conj(P), P))
        assert np.max(np.abs(G - np.eye(2 * nv))) < 1e-13
        for v in cands:
            assert np.max(np.abs(mg.prolong(P, blk, mg.restrict(P, blk, v)) - v)) < 1e-12
        rng = np.random.default_rng(seed)
        r = rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape)
        xc = rng.standard_normal(blk.coarse + (2 * nv,)) + 1j * rng.standard_normal(blk.coarse + (2 * nv,))
        lhs = np.vdot(mg.prolong(P, blk, xc), r)
        rhs = np.vdot(xc, mg.restrict(P, blk, r))
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))

    check()
