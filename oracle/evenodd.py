"""Oracle: even-odd (red-black) preconditioning of the Wilson-Dirac system, plain FP64 (test
infrastructure only).

The paper solves the full system D x = b.  Even-odd preconditioning is the
standard Schur-complement reduction of the same Sec. 1 operator, used here
for the fine-level smoother and the unpreconditioned Krylov baselines.

Sites split by parity p(n) = (x + y + z + t) mod 2.  With M = 4 + m and the
hopping term H of Sec. 1,
    D = M - 1/2 H,   H psi(n) = sum_mu [(1 - g_mu) U_mu(n) psi(n+mu) + (1 + g_mu) U_mu(n-mu)^+ psi(n-mu)],
H links only sites of opposite parity, so in (even, odd) blocks
    D = [[M, -1/2 H_eo], [-1/2 H_oe, M]]
and eliminating the odd sites leaves the Schur complement on the even sites
    S x_e = M x_e - 1/(4 M) H_eo H_oe x_e,
solved against  b^_e = b_e + 1/(2 M) H_eo b_o,  after which
    x_o = (b_o + 1/2 H_oe x_e) / M.
S inherits gamma5-Hermiticity from D: S^+ = gamma5 S gamma5.

Half-lattice fields ("even" or "odd" vectors) hold the sites of one parity
in lexicographic site order (x fastest): shape (V/2, 4, 3).  With Lx even the
k-th site of a parity has lexicographic index 2k or 2k + 1.

``eo_smooth`` is the fine-level smoother built on this: the Sec. 3 MR
smoother (omega, ``steps`` steps from zero) applied to the Schur system,
with the odd sites then solved exactly.  Its correction e satisfies
(r - D e)_o = 0, and (r - D e)_e is the Schur residual.

Only tests/, the package smoke check and the benchmark's CPU baseline import
this module.
"""
import numpy as np

from . import dirac
from .multigrid import mr_relax


def parity_masks(lattice):
    """Boolean (even, odd) masks over a (Lt, Lz, Ly, Lx) lattice."""
    t, z, y, x = np.indices(tuple(lattice))
    odd = ((t + z + y + x) % 2).astype(bool)
    return ~odd, odd


def split(psi):
    """(psi_e, psi_o): the even and odd sites of a (Lt, Lz, Ly, Lx, 4, 3) field, each (V/2, 4, 3)."""
    even, odd = parity_masks(psi.shape[:4])
    return psi[even], psi[odd]


def merge(psi_e, psi_o, lattice):
    """The full field whose even and odd sites are psi_e and psi_o."""
    even, odd = parity_masks(lattice)
    out = np.zeros(tuple(lattice) + (4, 3), dtype=np.complex128)
    out[even] = psi_e
    out[odd] = psi_o
    return out


def hopping(U, psi):
    """H psi.  D = (4 + m) - 1/2 H, so at m = -4 the Wilson operator is -1/2 H exactly."""
    return -2.0 * dirac.wilson_dirac(U, psi, -4.0)


def hop_eo(U, psi_o):
    """H_eo psi_o: the even sites of H applied to the field that is psi_o on the odd sites, 0 elsewhere."""
    lat = U.shape[1:5]
    return split(hopping(U, merge(np.zeros_like(psi_o), psi_o, lat)))[0]


def hop_oe(U, psi_e):
    """H_oe psi_e: the odd sites of H applied to the field that is psi_e on the even sites, 0 elsewhere."""
    lat = U.shape[1:5]
    return split(hopping(U, merge(psi_e, np.zeros_like(psi_e), lat)))[1]


def schur(U, mass, x_e):
    """S x_e = M x_e - 1/(4 M) H_eo H_oe x_e, M = 4 + mass."""
    M = 4.0 + mass
    return M * x_e - hop_eo(U, hop_oe(U, x_e)) / (4.0 * M)


def schur_rhs(U, mass, b):
    """b^_e = b_e + 1/(2 M) H_eo b_o for a full right-hand side b."""
    M = 4.0 + mass
    b_e, b_o = split(b)
    return b_e + hop_eo(U, b_o) / (2.0 * M)


def reconstruct(U, mass, b, x_e):
    """The full solution from the even one: x_o = (b_o + 1/2 H_oe x_e) / M."""
    M = 4.0 + mass
    _, b_o = split(b)
    x_o = (b_o + 0.5 * hop_oe(U, x_e)) / M
    return merge(x_e, x_o, U.shape[1:5])


def eo_solve(U, mass, b, solve_even):
    """x = D^-1 b through the Schur system; solve_even(apply_S, b^_e) returns x_e."""
    x_e = solve_even(lambda v: schur(U, mass, v), schur_rhs(U, mass, b))
    return reconstruct(U, mass, b, x_e)


def eo_smooth(U, mass, r, steps, omega=0.8):
    """Even-odd smoother for D e = r (fields (Lt, Lz, Ly, Lx, 4, 3)): ``steps`` MR steps on the Schur
    system from e_e = 0, then the exact odd-site solve.  Returns (e, r - D e)."""
    e_e, _ = mr_relax(lambda v: schur(U, mass, v), schur_rhs(U, mass, r), None, steps, omega)
    e = reconstruct(U, mass, r, e_e)
    return e, r - dirac.wilson_dirac(U, e, mass)
