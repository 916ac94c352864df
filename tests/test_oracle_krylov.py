"""Pins of the oracle's unpreconditioned Krylov baselines (the comparison solvers of Secs. 4-5).

* both reach the dense-LU solution of the Wilson system on 4^4;
* BiCGstab's iterates equal those of scipy's independent BiCGstab (the same
  published method, shadow residual r0) while rounding allows;
* CGNR's iterates equal scipy's CG applied to D^+ D x = D^+ b, with D^+ built
  from gamma5-Hermiticity (Sec. 1);
* a multiple of the identity is solved by BiCGstab in one iteration.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse.linalg as sla

from oracle import dirac
from oracle import krylov
from paper_0811_4331_gb300 import inputs


def _system(dims=(4, 4, 4, 4), m=0.1, seed=0):
    U = inputs.random_gauge(dims, seed)
    lat = (dims[3], dims[2], dims[1], dims[0])
    shp = lat + (4, 3)

    def A(v):
        return dirac.wilson_dirac(U, v.reshape(shp), m).reshape(v.shape)

    def Ad(v):
        return dirac.apply_gamma5(dirac.wilson_dirac(U, dirac.apply_gamma5(v.reshape(shp)), m)).reshape(v.shape)

    b = inputs.gaussian_spinor(dims, 1).reshape(-1)
    return A, Ad, b, shp


def test_bicgstab_and_cgnr_reach_the_lu_solution():
    A, Ad, b, shp = _system()
    D = dirac.dense_matrix(A, (b.size,))
    xl = scipy.linalg.solve(D, b)
    x, info = krylov.bicgstab(A, b, tol=1e-10)
    assert info["true_rel_residual"] <= 1e-10
    assert np.linalg.norm(x - xl) < 1e-8 * np.linalg.norm(xl)
    x2, info2 = krylov.cgnr(A, Ad, b, tol=1e-10)
    assert info2["true_rel_residual"] <= 1e-10
    assert np.linalg.norm(x2 - xl) < 1e-8 * np.linalg.norm(xl)
    assert info2["iters"] > info["iters"]  # the normal equations square the condition number


def test_iterates_match_independent_implementations():
    A, Ad, b, shp = _system(dims=(2, 2, 2, 4), m=0.3, seed=2)
    n = b.size
    op = sla.LinearOperator((n, n), matvec=A, dtype=np.complex128)
    ref, mine = [], []
    sla.bicgstab(op, b, rtol=1e-300, atol=0.0, maxiter=6, callback=lambda xk: ref.append(xk.copy()))
    try:
        krylov.bicgstab(A, b, tol=1e-300, max_iter=6, callback=lambda xk: mine.append(xk.copy()))
    except ArithmeticError:
        pass
    assert len(ref) >= 5 and len(mine) >= 5
    for k in range(5):
        assert np.linalg.norm(mine[k] - ref[k]) < 1e-10 * np.linalg.norm(ref[k]), k
    N = sla.LinearOperator((n, n), matvec=lambda v: Ad(A(v)), dtype=np.complex128)
    ref, mine = [], []
    sla.cg(N, Ad(b), rtol=1e-300, atol=0.0, maxiter=6, callback=lambda xk: ref.append(xk.copy()))
    try:
        krylov.cgnr(A, Ad, b, tol=1e-300, max_iter=6, callback=lambda xk: mine.append(xk.copy()))
    except ArithmeticError:
        pass
    for k in range(5):
        assert np.linalg.norm(mine[k] - ref[k]) < 1e-10 * np.linalg.norm(ref[k]), k


def test_identity_is_one_iteration():
    b = np.arange(1, 7) + 1j * np.arange(6)
    x, info = krylov.bicgstab(lambda v: 2.5 * v, b, tol=1e-12)
    assert info["iters"] == 1
    assert np.allclose(x, b / 2.5, rtol=1e-14)


def test_methods_reach_the_dense_solution_on_random_shapes():
    """BiCGstab and CGNR against a dense solve over random small lattices (extents 1..3), masses and fields."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=6, deadline=None, derandomize=True)
    @hyp.given(dims=st.tuples(*[st.integers(1, 3)] * 4), m=st.floats(0.05, 1.0), seed=st.integers(0, 1000))
    def check(dims, m, seed):
        A, Ad, b, shp = _system(dims, m, seed)
        D = dirac.dense_matrix(A, (b.size,))
        xl = np.linalg.solve(D, b)
        for x, info in (krylov.bicgstab(A, b, tol=1e-11), krylov.cgnr(A, Ad, b, tol=1e-11)):
            assert info["true_rel_residual"] <= 1e-11
            assert np.linalg.norm(D @ x - b) <= 1.01e-11 * np.linalg.norm(b)
            assert np.linalg.norm(x - xl) <= 1e-7 * np.linalg.norm(xl)

    check()
