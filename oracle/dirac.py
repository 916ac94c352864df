"""Oracle: the 4D SU(3) Wilson-Dirac operator in FP64 (test infrastructure only).

Sec. 1 (Eq. 1.1 and the paragraph after it) defines D = Dslash + m with
Dslash built from central covariant differences times the Dirac gamma
matrices, plus a second-order Wilson term.  With lattice spacing 1 and Wilson
parameter r = 1 this is, for a spinor psi(n) with 4 spin x 3 colour components,

  (D psi)(n) = (4 + m) psi(n)
               - 1/2 sum_mu [ (1 - gamma_mu) U_mu(n)        psi(n + mu)
                            + (1 + gamma_mu) U_mu(n - mu)^+ psi(n - mu) ].

Readings where the paper is silent:
  * gamma basis: the chiral basis
        gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1, 2, 3  <->  x, y, z)
        gamma_4 = [[0, 1], [1, 0]]                  (t)
    so gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1): spins
    {0, 1} carry chirality +1 and spins {2, 3} chirality -1.
  * r = 1, spacing 1, periodic boundaries in all four directions; the (4 + m)
    diagonal puts the free critical mass at m = 0 and the interacting one near
    the m_crit = -0.8049 quoted for beta = 6.0 in Sec. 5.

Array conventions (numpy, C order): a fine spinor field has shape
(Lt, Lz, Ly, Lx, 4, 3) -- site index lexicographic with x fastest, then spin,
then colour; a gauge field has shape (4, Lt, Lz, Ly, Lx, 3, 3) with mu = 0..3
for x, y, z, t.  Direction mu moves along array axis 3 - mu.
"""
import numpy as np

_SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def gamma_matrices():
    """The four Euclidean Dirac matrices (x, y, z, t) in the chiral basis."""
    g = []
    for k in range(3):
        g.append(np.block([[_Z2, -1j * _SIGMA[k]], [1j * _SIGMA[k], _Z2]]))
    g.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
    return np.array(g)


GAMMA = gamma_matrices()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
IDENTITY4 = np.eye(4, dtype=np.complex128)


def axis_of(mu):
    """Array axis of direction mu in a (Lt, Lz, Ly, Lx, ...) field."""
    return 3 - mu


def shift(field, mu, step):
    """field(n + step * mu) as an array over n, with periodic wrap."""
    return np.roll(field, -step, axis=axis_of(mu))


def colour_mul(U, psi):
    """sum_b U[..., a, b] psi[..., s, b] at every site."""
    return np.einsum("...ab,...sb->...sa", U, psi)


def spin_mul(G, psi):
    """sum_t G[s, t] psi[..., t, a] at every site."""
    return np.einsum("st,...ta->...sa", G, psi)


def wilson_dirac(U, psi, mass):
    """(D psi) for the Wilson-Dirac operator written out above (Sec. 1)."""
    out = (4.0 + mass) * psi
    for mu in range(4):
        forward = colour_mul(U[mu], shift(psi, mu, +1))
        U_back = shift(U[mu], mu, -1)
        backward = colour_mul(np.conj(np.swapaxes(U_back, -1, -2)), shift(psi, mu, -1))
        out = out - 0.5 * (spin_mul(IDENTITY4 - GAMMA[mu], forward)
                           + spin_mul(IDENTITY4 + GAMMA[mu], backward))
    return out


def apply_gamma5(psi):
    """gamma_5 psi (diag(1, 1, -1, -1) in spin)."""
    return spin_mul(GAMMA5, psi)


def dense_matrix(apply, shape):
    """Dense matrix of a linear map on fields of ``shape``, column by column (any output size)."""
    n = int(np.prod(shape))
    e = np.zeros(n, dtype=np.complex128)
    cols = []
    for j in range(n):
        e[j] = 1.0
        cols.append(np.asarray(apply(e.reshape(shape))).reshape(-1))
        e[j] = 0.0
    return np.stack(cols, axis=1)


# --------------------------------------------------------------------------
# 9-point stencil form of D.  Direction index d: 0 = the site itself,
# 1 + 2 mu = the hop to n + mu, 2 + 2 mu = the hop to n - mu.  An operator in
# stencil form is (A y)(n) = sum_d A_d(n) y(n + e_d), where A_d(n) is an
# ncomp x ncomp matrix.  For the fine level ncomp = 12 with component index
# spin * 3 + colour.
# --------------------------------------------------------------------------

def stencil_offset(d):
    """(mu, step) of stencil direction d >= 1."""
    return (d - 1) // 2, (+1 if d % 2 == 1 else -1)


def wilson_stencil(U, mass):
    """Blocks A_d(n) of D as an array of shape (9, Lt, Lz, Ly, Lx, 12, 12).

    A_0 = (4 + m) 1, A_{+mu}(n) = -1/2 (1 - gamma_mu) (x) U_mu(n),
    A_{-mu}(n) = -1/2 (1 + gamma_mu) (x) U_mu(n - mu)^+  (Sec. 1).
    """
    lat = U.shape[1:5]
    A = np.zeros((9,) + lat + (12, 12), dtype=np.complex128)
    A[0] = (4.0 + mass) * np.eye(12)
    for mu in range(4):
        U_back = np.conj(np.swapaxes(shift(U[mu], mu, -1), -1, -2))
        A[1 + 2 * mu] = -0.5 * np.einsum("st,...ab->...satb", IDENTITY4 - GAMMA[mu],
                                         U[mu]).reshape(lat + (12, 12))
        A[2 + 2 * mu] = -0.5 * np.einsum("st,...ab->...satb", IDENTITY4 + GAMMA[mu],
                                         U_back).reshape(lat + (12, 12))
    return A


def stencil_apply(A, y):
    """(A y)(n) = sum_d A_d(n) y(n + e_d) for y of shape (Lt, Lz, Ly, Lx, ncomp)."""
    out = np.einsum("...ij,...j->...i", A[0], y)
    for d in range(1, 9):
        mu, step = stencil_offset(d)
        out = out + np.einsum("...ij,...j->...i", A[d], shift(y, mu, step))
    return out


def wilson_dirac_site(U, psi, mass, site):
    """(D psi)(n) at one site n = (x, y, z, t), from the same definition (Sec. 1).

    Used to check sampled outputs of lattices too large for the whole-field
    oracle.  Neighbour coordinates wrap periodically.
    """
    Lt, Lz, Ly, Lx = psi.shape[:4]
    L = (Lx, Ly, Lz, Lt)
    x = list(site)

    def at(c):
        return (c[3] % L[3], c[2] % L[2], c[1] % L[1], c[0] % L[0])

    out = (4.0 + mass) * psi[at(x)]
    for mu in range(4):
        up = list(x)
        up[mu] += 1
        dn = list(x)
        dn[mu] -= 1
        fwd = psi[at(up)] @ U[mu][at(x)].T               # U_mu(n) psi(n + mu), colour on the right
        bwd = psi[at(dn)] @ np.conj(U[mu][at(dn)])       # U_mu(n - mu)^+ psi(n - mu)
        out = out - 0.5 * ((IDENTITY4 - GAMMA[mu]) @ fwd + (IDENTITY4 + GAMMA[mu]) @ bwd)
    return out
