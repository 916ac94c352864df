"""Pins of the oracle Wilson-Dirac operator against facts the paper and mathematics fix.

Each test checks oracle.dirac against something other than itself:
closed forms (free-field plane waves and spectrum), algebraic identities the
paper states (gamma5-Hermiticity, Sec. 1), gauge covariance, and a dense LU
solve.  A dropped term, a sign error, U in place of U^+, a wrong neighbour
index or a wrong gamma basis fails at least one of them.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import dirac
from paper_0811_4331_gb300 import inputs


def _lat(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx)


def test_gamma_clifford_and_chiral_basis():
    G = dirac.GAMMA
    for mu in range(4):
        assert np.allclose(G[mu], G[mu].conj().T)  # Euclidean gammas are Hermitian
        for nu in range(4):
            anti = G[mu] @ G[nu] + G[nu] @ G[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=0)
    # chiral basis reading: gamma5 = gamma1 gamma2 gamma3 gamma4 = diag(1, 1, -1, -1)
    assert np.array_equal(dirac.GAMMA5, np.diag([1, 1, -1, -1]).astype(complex))


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (3, 4, 2, 5)])
def test_free_field_plane_waves(dims):
    """U = 1: D e^{ip.n} u = e^{ip.n} [m + sum(1 - cos p) + i sum gamma_mu sin p_mu] u."""
    m = 0.137
    U = inputs.unit_gauge(dims)
    lat = _lat(dims)
    t, z, y, x = np.meshgrid(*[np.arange(L) for L in lat], indexing="ij")
    rng = np.random.default_rng(5)
    for _ in range(6):
        k = [rng.integers(0, L) for L in dims]
        p = 2 * np.pi * np.array(k) / np.array(dims)
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = phase[..., None, None] * u
        Dp = (m + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(
            np.array(dirac.GAMMA[mu]) * np.sin(p[mu]) for mu in range(4))
        expect = phase[..., None, None] * (Dp @ u)
        assert np.max(np.abs(dirac.wilson_dirac(U, psi, m) - expect)) < 1e-13


def test_free_field_spectrum():
    """Closed-form spectrum m + sum(1 - cos p) +- i sqrt(sum sin^2 p), each 6-fold."""
    dims = (2, 2, 2, 4)
    m = 0.1
    U = inputs.unit_gauge(dims)
    lat = _lat(dims)
    D = dirac.dense_matrix(lambda y: dirac.wilson_dirac(U, y, m), lat + (4, 3))
    ev = np.linalg.eigvals(D)
    expect = []
    for k in np.ndindex(*dims):
        p = 2 * np.pi * np.array(k) / np.array(dims)
        re = m + np.sum(1 - np.cos(p))
        im = np.sqrt(np.sum(np.sin(p) ** 2))
        expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    expect = np.array(expect)
    # greedy multiset match
    left = list(ev)
    for e in expect:
        j = int(np.argmin(np.abs(np.array(left) - e)))
        assert abs(left[j] - e) < 1e-10
        left.pop(j)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 3, 4, 5)])
def test_gamma5_hermiticity(dims):
    """D^+ = gamma5 D gamma5 (Sec. 1): <y, g5 D x> = conj <x, g5 D y>."""
    m = -0.3
    U = inputs.random_gauge(dims, 11)
    x = inputs.gaussian_spinor(dims, 1)
    y = inputs.gaussian_spinor(dims, 2)

    def g5D(v):
        return dirac.apply_gamma5(dirac.wilson_dirac(U, v, m))

    a = np.vdot(y, g5D(x))
    b = np.conj(np.vdot(x, g5D(y)))
    assert abs(a - b) <= 1e-13 * abs(a)
    # and it is not trivially true for D itself (D is non-Hermitian, Sec. 1)
    a2 = np.vdot(y, dirac.wilson_dirac(U, x, m))
    b2 = np.conj(np.vdot(x, dirac.wilson_dirac(U, y, m)))
    assert abs(a2 - b2) > 1e-3 * abs(a2)


def test_gauge_covariance():
    """U_mu(n) -> G(n) U_mu(n) G(n+mu)^+, psi -> G psi  gives  D' (G psi) = G (D psi)."""
    dims = (4, 2, 3, 4)
    m = 0.05
    U = inputs.random_gauge(dims, 3)
    lat = _lat(dims)
    rng = np.random.default_rng(9)
    G = inputs.random_su3(rng, int(np.prod(lat)), 1.0).reshape(lat + (3, 3))
    Ug = np.empty_like(U)
    for mu in range(4):
        Gp = dirac.shift(G, mu, +1)
        Ug[mu] = G @ U[mu] @ np.conj(np.swapaxes(Gp, -1, -2))
    psi = inputs.gaussian_spinor(dims, 4)
    Gpsi = np.einsum("...ab,...sb->...sa", G, psi)
    lhs = dirac.wilson_dirac(Ug, Gpsi, m)
    rhs = np.einsum("...ab,...sb->...sa", G, dirac.wilson_dirac(U, psi, m))
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(rhs))


def test_constant_mode_free_field():
    """U = 1, constant spinor: only the mass survives (p = 0 plane wave)."""
    dims = (3, 3, 2, 2)
    U = inputs.unit_gauge(dims)
    psi = np.ones(_lat(dims) + (4, 3), dtype=complex) * (0.3 - 0.7j)
    assert np.max(np.abs(dirac.wilson_dirac(U, psi, 0.25) - 0.25 * psi)) < 1e-15


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 2, 5, 2)])
def test_stencil_form_equals_operator(dims):
    U = inputs.random_gauge(dims, 6)
    psi = inputs.gaussian_spinor(dims, 7)
    lat = _lat(dims)
    A = dirac.wilson_stencil(U, 0.2)
    got = dirac.stencil_apply(A, psi.reshape(lat + (12,))).reshape(psi.shape)
    assert np.max(np.abs(got - dirac.wilson_dirac(U, psi, 0.2))) < 1e-13


def test_dense_lu_solve_2x4():
    """Dense LU (library routine) on a 2^4 lattice: ||D x - b|| / ||b|| <= 1e-13."""
    dims = (2, 2, 2, 2)
    U = inputs.random_gauge(dims, 0)
    lat = _lat(dims)
    m = 0.1
    D = dirac.dense_matrix(lambda y: dirac.wilson_dirac(U, y, m), lat + (4, 3))
    b = inputs.gaussian_spinor(dims, 1)
    x = scipy.linalg.lu_solve(scipy.linalg.lu_factor(D), b.reshape(-1)).reshape(b.shape)
    r = b - dirac.wilson_dirac(U, x, m)
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(b)
    # Re(lambda) > 0 for this field and mass (Sec. 1)
    assert np.min(np.linalg.eigvals(D).real) > 0


def test_single_site_operator_matches_field_operator():
    dims = (3, 4, 2, 5)
    U = inputs.random_gauge(dims, 1)
    psi = inputs.gaussian_spinor(dims, 2)
    full = dirac.wilson_dirac(U, psi, 0.3)
    for site in [(0, 0, 0, 0), (2, 3, 1, 4), (1, 0, 1, 2), (2, 0, 0, 0)]:
        x, y, z, t = site
        assert np.max(np.abs(dirac.wilson_dirac_site(U, psi, 0.3, site) - full[t, z, y, x])) < 1e-13


def test_covariance_and_gamma5_hermiticity_on_random_shapes():
    """Gauge covariance and gamma5-Hermiticity over random extents 1..5 (odd, even, length 1), masses and
    fields: a wrong hop direction, link index or boundary wrap breaks one of the two."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=8, deadline=None, derandomize=True)
    @hyp.given(dims=st.tuples(*[st.integers(1, 5)] * 4), m=st.floats(-1.0, 1.0), seed=st.integers(0, 10 ** 6))
    def check(dims, m, seed):
        U = inputs.random_gauge(dims, seed)
        lat = _lat(dims)
        rng = np.random.default_rng(seed + 1)
        G = inputs.random_su3(rng, int(np.prod(lat)), 1.0).reshape(lat + (3, 3))
        Ug = np.empty_like(U)
        for mu in range(4):
            Ug[mu] = G @ U[mu] @ np.conj(np.swapaxes(dirac.shift(G, mu, +1), -1, -2))
        x = inputs.gaussian_spinor(dims, seed + 2)
        y = inputs.gaussian_spinor(dims, seed + 3)
        Gx = np.einsum("...ab,...sb->...sa", G, x)
        lhs = dirac.wilson_dirac(Ug, Gx, m)
        rhs = np.einsum("...ab,...sb->...sa", G, dirac.wilson_dirac(U, x, m))
        assert np.max(np.abs(lhs - rhs)) <= 1e-12 * max(1.0, np.max(np.abs(rhs)))
        a = np.vdot(y, dirac.apply_gamma5(dirac.wilson_dirac(U, x, m)))
        b = np.vdot(x, dirac.apply_gamma5(dirac.wilson_dirac(U, y, m)))
        assert abs(a - np.conj(b)) <= 1e-12 * max(1.0, abs(a))

    check()
