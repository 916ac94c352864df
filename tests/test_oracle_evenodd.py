"""Pins of the oracle's even-odd (Schur-complement) reduction of the Wilson system.

Each pin fixes the result by something other than the formula it checks:

* the half-lattice order is the lexicographic order of each parity (the
  k-th site of a parity sits at lexicographic index 2k or 2k + 1);
* S equals the block Schur complement D_ee - D_eo D_oo^-1 D_oe of the dense
  Wilson matrix, with the blocks cut out by parity (catches a wrong factor,
  sign or parity assignment in either hop);
* solving the Schur system densely and reconstructing the odd sites gives
  the dense solution of D x = b (pins b^_e and the odd-site solve);
* gamma5 S is Hermitian (gamma5-Hermiticity survives the reduction);
* free field, constant spinor: H psi = 8 psi, so S psi = (M - 16/M) psi, and
  S has the zero mode of D at m = 0;
* the even-odd smoother leaves no residual on odd sites, reduces to
  e = (0, r_o / M) with no MR step, and converges to D^-1 r;
* MG-GCR with the even-odd fine smoother reaches the tolerance.
"""
import numpy as np
import pytest

from oracle import dirac, evenodd, krylov
from oracle import multigrid as mg
from paper_0811_4331_gb300 import inputs


def _lat(dims):
    return (dims[3], dims[2], dims[1], dims[0])


def test_half_lattice_order():
    dims = (4, 2, 2, 4)
    lat = _lat(dims)
    idx = np.arange(int(np.prod(lat))).reshape(lat)
    even, odd = evenodd.parity_masks(lat)
    for mask in (even, odd):
        lex = idx[mask]
        assert lex.size == idx.size // 2
        assert np.all(lex // 2 == np.arange(lex.size))
    psi = inputs.gaussian_spinor(dims, 3)
    e, o = evenodd.split(psi)
    assert np.array_equal(evenodd.merge(e, o, lat), psi)


def _dense_blocks(U, m):
    lat = U.shape[1:5]
    shp = lat + (4, 3)
    D = dirac.dense_matrix(lambda v: dirac.wilson_dirac(U, v, m), shp)
    even, _ = evenodd.parity_masks(lat)
    dof_even = np.repeat(even.reshape(-1), 12)
    return D, dof_even


@pytest.mark.parametrize("m", [0.3, -0.7])
def test_schur_complement_equals_the_dense_block_elimination(m):
    dims = (4, 2, 2, 4)
    U = inputs.random_gauge(dims, 2)
    D, de = _dense_blocks(U, m)
    Dee, Deo = D[np.ix_(de, de)], D[np.ix_(de, ~de)]
    Doe, Doo = D[np.ix_(~de, de)], D[np.ix_(~de, ~de)]
    S_blocks = Dee - Deo @ np.linalg.solve(Doo, Doe)
    half = (de.sum() // 12, 4, 3)
    S = dirac.dense_matrix(lambda v: evenodd.schur(U, m, v), half)
    assert np.max(np.abs(S - S_blocks)) < 1e-12
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), half[0])
    G5S = g5[:, None] * S
    assert np.max(np.abs(G5S - G5S.conj().T)) < 1e-12


def test_schur_solve_reconstructs_the_dense_solution():
    dims = (4, 2, 2, 4)
    m = 0.1
    U = inputs.random_gauge(dims, 4)
    D, _ = _dense_blocks(U, m)
    b = inputs.gaussian_spinor(dims, 5)
    want = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)

    def dense_even_solve(apply_S, bh):
        S = dirac.dense_matrix(apply_S, bh.shape)
        return np.linalg.solve(S, bh.reshape(-1)).reshape(bh.shape)

    got = evenodd.eo_solve(U, m, b, dense_even_solve)
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))


def test_free_field_constant_spinor():
    dims = (4, 4, 2, 2)
    lat = _lat(dims)
    U = np.zeros((4,) + lat + (3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    u = inputs.gaussian_spinor((1, 1, 1, 1), 9).reshape(4, 3)
    psi = np.broadcast_to(u, lat + (4, 3)).copy()
    assert np.max(np.abs(evenodd.hopping(U, psi) - 8.0 * psi)) < 1e-13
    psi_e, _ = evenodd.split(psi)
    for m in (0.5, 0.0, -0.2):
        M = 4.0 + m
        assert np.max(np.abs(evenodd.schur(U, m, psi_e) - (M - 16.0 / M) * psi_e)) < 1e-12
    assert np.max(np.abs(evenodd.schur(U, 0.0, psi_e))) < 1e-12


def test_even_odd_smoother():
    dims = (4, 4, 4, 4)
    m = 0.5
    U = inputs.random_gauge(dims, 6)
    r = inputs.gaussian_spinor(dims, 7)
    e0, res0 = evenodd.eo_smooth(U, m, r, 0)
    r_e, r_o = evenodd.split(r)
    assert np.array_equal(evenodd.split(e0)[0], np.zeros_like(r_e))
    assert np.max(np.abs(evenodd.split(e0)[1] - r_o / 4.5)) < 1e-15
    prev = np.linalg.norm(res0)
    for steps in (2, 8):
        e, res = evenodd.eo_smooth(U, m, r, steps)
        assert np.max(np.abs(evenodd.split(res)[1])) < 1e-12 * np.max(np.abs(r))
        assert np.linalg.norm(res) < prev
        prev = np.linalg.norm(res)
    e, res = evenodd.eo_smooth(U, m, r, 200, omega=1.0)
    x, _ = krylov.bicgstab(lambda v: dirac.wilson_dirac(U, v, m), r, tol=1e-13)
    assert np.linalg.norm(e - x) < 1e-9 * np.linalg.norm(x)


def test_mg_gcr_with_the_even_odd_smoother_converges():
    dims = (4, 4, 4, 4)
    m = -0.3
    U = inputs.random_gauge(dims, 8)
    lat = _lat(dims)
    starts = [inputs.gaussian_spinor(dims, 100 + k).reshape(lat + (12,)) for k in range(8)]
    levels = [dict(block=(2, 2, 2, 2), nv=8, sweeps=6)]
    b = inputs.gaussian_spinor(dims, 11).reshape(lat + (12,))
    its = {}
    for sm in ("mr", "eo"):
        hier = mg.mg_setup(U, m, levels, [starts], fine_smoother=sm)
        x, info = mg.mg_solve(hier, b, tol=1e-10)
        r = b - hier[0].apply(x)
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
        its[sm] = info["iters"]
    assert its["eo"] <= its["mr"] + 2, its


def test_schur_identity_on_random_shapes():
    """The block-elimination pin over random even extents (2 or 4 per direction), masses and fields."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=6, deadline=None, derandomize=True)
    @hyp.given(ext=st.tuples(*[st.sampled_from([2, 4])] * 4).filter(lambda e: e[0] * e[1] * e[2] * e[3] <= 64),
               m=st.floats(-0.9, 0.9), seed=st.integers(0, 1000))
    def check(ext, m, seed):
        U = inputs.random_gauge(ext, seed)
        D, de = _dense_blocks(U, m)
        S_blocks = D[np.ix_(de, de)] - D[np.ix_(de, ~de)] @ np.linalg.solve(D[np.ix_(~de, ~de)], D[np.ix_(~de, de)])
        half = (de.sum() // 12, 4, 3)
        S = dirac.dense_matrix(lambda v: evenodd.schur(U, m, v), half)
        assert np.max(np.abs(S - S_blocks)) < 1e-11 * max(1.0, np.max(np.abs(S_blocks)))

    check()
