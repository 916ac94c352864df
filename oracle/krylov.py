"""Oracle: the unpreconditioned Krylov solvers the paper compares multigrid with (test infrastructure only).

Sec. 4 and Sec. 5 of the paper measure MG against plain BiCGstab on the
Wilson system (and CG in the 2d study).  Both are textbook methods:

* ``bicgstab`` -- BiCGstab of van der Vorst (SIAM J. Sci. Stat. Comput. 13,
  1992) on D x = b, shadow residual = the initial residual, stopping on the
  half step when s is already small;
* ``cgnr``     -- conjugate gradients on the normal equations
  D^+ D x = D^+ b (Hestenes-Stiefel CG applied to the Hermitian positive
  definite D^+ D), with D^+ = gamma5 D gamma5 (gamma5-Hermiticity, Sec. 1).

Both stop when the recursively updated residual reaches tol ||b||, then
recompute the true residual b - D x; if it is above tol they continue from
the true residual (a restart).  Inner products <a|b> = sum conj(a) b.
Only tests/, the package smoke check and the benchmark's CPU baseline import
this module.
"""
import numpy as np

from .multigrid import inner, norm2


def bicgstab(apply, b, tol=1e-10, max_iter=100000, callback=None):
    """Returns (x, info) with info = {"iters", "matvecs", "true_rel_residual"}; callback(x) after
    every iteration."""
    bn = np.sqrt(norm2(b))
    x = np.zeros_like(b)
    r = b.copy()
    iters = matvecs = 0
    while iters < max_iter:
        rhat = r.copy()
        rho = alpha = omega = 1.0 + 0j
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        while iters < max_iter:
            rho_new = inner(rhat, r)
            beta = (rho_new / rho) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = apply(p)
            alpha = rho_new / inner(rhat, v)
            s = r - alpha * v
            matvecs += 1
            iters += 1
            if np.sqrt(norm2(s)) <= tol * bn:  # converged on the half step
                x = x + alpha * p
                r = s
                if callback:
                    callback(x)
                break
            t = apply(s)
            matvecs += 1
            omega = inner(t, s) / inner(t, t)
            x = x + alpha * p + omega * s
            r = s - omega * t
            rho = rho_new
            if callback:
                callback(x)
            if np.sqrt(norm2(r)) <= tol * bn:
                break
        r = b - apply(x)
        matvecs += 1
        true = np.sqrt(norm2(r)) / bn
        if true <= tol:
            return x, {"iters": iters, "matvecs": matvecs, "true_rel_residual": true}
    raise ArithmeticError("BiCGstab did not converge")


def cgnr(apply, apply_dag, b, tol=1e-10, max_iter=100000, callback=None):
    """CG on D^+ D x = D^+ b; the stopping test is on the residual of D x = b; callback(x) after every
    iteration."""
    bn = np.sqrt(norm2(b))
    x = np.zeros_like(b)
    iters = matvecs = 0
    r = b.copy()
    while iters < max_iter:
        z = apply_dag(r)  # residual of the normal equations
        matvecs += 1
        p = z.copy()
        zz = norm2(z)
        while iters < max_iter:
            q = apply(p)
            matvecs += 1
            a = zz / norm2(q)
            x = x + a * p
            r = r - a * q
            iters += 1
            if callback:
                callback(x)
            if np.sqrt(norm2(r)) <= tol * bn:
                break
            z = apply_dag(r)
            matvecs += 1
            zz_new = norm2(z)
            p = z + (zz_new / zz) * p
            zz = zz_new
        r = b - apply(x)
        matvecs += 1
        true = np.sqrt(norm2(r)) / bn
        if true <= tol:
            return x, {"iters": iters, "matvecs": matvecs, "true_rel_residual": true}
    raise ArithmeticError("CGNR did not converge")
