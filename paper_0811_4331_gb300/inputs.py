"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds none of the solver's arithmetic (no Dirac operator, no
multigrid, no Krylov step).  It generates:

* SU(3) gauge fields U = exp(i eps H) with H a Gaussian traceless Hermitian
  3x3 matrix per link (eps = 0.3 for the small 4^4 workload);
* Wilson-action (beta = 6.0) gauge fields by Cabibbo-Marinari heatbath over
  the three SU(2) subgroups, each updated with the Kennedy-Pendleton
  algorithm (Phys. Lett. B 156 (1985) 393), from a cold start, reunitarised
  after every sweep;
* Gaussian and point-source right-hand sides;
* random starting vectors for the null-vector relaxation, from a
  counter-based generator: element i of a stream with 64-bit seed s uses the
  SplitMix64 outputs number 2i and 2i+1 of state s (Steele, Lea, Flood,
  OOPSLA 2014: output m = mix(s + (m + 1) * 0x9E3779B97F4A7C15)), each
  turned into a uniform u in (0, 1] as ((x >> 11) + 1) * 2^-53, and the pair
  into one complex Gaussian by Box-Muller:
  sqrt(-2 ln u1) * (cos(2 pi u2) + i sin(2 pi u2)).  The library's
  on-device generator implements the same definition.

Layouts are the external ones of the C ABI: a spinor field is
(Lt, Lz, Ly, Lx, 4, 3) complex128 (x fastest, then spin, then colour); a gauge
field is (4, Lt, Lz, Ly, Lx, 3, 3) with mu = 0..3 for x, y, z, t.  ``dims`` is
always given as (Lx, Ly, Lz, Lt).
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _shape(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx)


def splitmix64(seed, m):
    """Output number m (uint64 array) of SplitMix64 started from state ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(m, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def counter_gaussian(seed, n, offset=0):
    """Complex Gaussians number offset .. offset+n-1 of stream ``seed`` (definition above)."""
    i = np.arange(offset, offset + n, dtype=np.uint64)
    x1 = splitmix64(seed, np.uint64(2) * i)
    x2 = splitmix64(seed, np.uint64(2) * i + np.uint64(1))
    u1 = ((x1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = ((x2 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2.0 * np.pi * u2) + 1j * rad * np.sin(2.0 * np.pi * u2)


def null_vector_starts(lattice_shape, ncomp, nv, seed):
    """``nv`` random start vectors of shape lattice_shape + (ncomp,) from stream ``seed``.

    Vector k element (site, comp) is stream element k * V * ncomp + site * ncomp + comp.
    """
    V = int(np.prod(lattice_shape))
    g = counter_gaussian(seed, nv * V * ncomp)
    return [g[k * V * ncomp:(k + 1) * V * ncomp].reshape(tuple(lattice_shape) + (ncomp,))
            for k in range(nv)]


# ------------------------------------------------------------------ gauge fields

def random_su3(rng, n, eps):
    """n matrices exp(i eps H), H = (A + A^+)/2 - tr/3, A Gaussian complex."""
    A = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real
    H = H - (tr / 3.0)[:, None, None] * np.eye(3)
    lam, Q = np.linalg.eigh(H)
    return np.einsum("nab,nb,ncb->nac", Q, np.exp(1j * eps * lam), np.conj(Q))


def random_gauge(dims, seed, eps=0.3):
    """Gauge field with U = exp(i eps H) on every link (mu-major, then site)."""
    rng = np.random.default_rng(seed)
    lat = _shape(dims)
    V = int(np.prod(lat))
    return random_su3(rng, 4 * V, eps).reshape((4,) + lat + (3, 3))


def random_gauge_fast(dims, seed, eps=0.3):
    """SU(3) field reunitarize(1 + eps (A - A^+)/2) with A Gaussian complex.

    A cheap generator for lattices where the eigen-decomposition of every
    link would take minutes; used where only the memory traffic of the
    operator matters, not the distribution of the links.
    """
    rng = np.random.default_rng(seed)
    lat = _shape(dims)
    shp = (4,) + lat + (3, 3)
    A = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    M = np.eye(3) + 0.5 * eps * (A - np.conj(np.swapaxes(A, -1, -2)))
    return reunitarize(M)


def unit_gauge(dims):
    lat = _shape(dims)
    U = np.zeros((4,) + lat + (3, 3), dtype=np.complex128)
    U[..., :, :] = np.eye(3)
    return U


def reunitarize(U):
    """Project onto SU(3): Gram-Schmidt the first two rows, third = conj(row0 x row1)."""
    r0 = U[..., 0, :]
    r0 = r0 / np.sqrt(np.sum(np.abs(r0) ** 2, axis=-1, keepdims=True))
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1, keepdims=True))
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def _roll(f, mu, step):
    # f(n + step * mu) for f shaped (Lt, Lz, Ly, Lx, ...)
    return np.roll(f, -step, axis=3 - mu)


def staple_sum(U, mu):
    """Sum over nu != mu of the up and down staples attached to U_mu(n)."""
    A = np.zeros_like(U[mu])
    for nu in range(4):
        if nu == mu:
            continue
        Unu_xmu = _roll(U[nu], mu, +1)
        A += Unu_xmu @ _dag(_roll(U[mu], nu, +1)) @ _dag(U[nu])
        Unu_xmu_mnu = _roll(Unu_xmu, nu, -1)
        A += _dag(Unu_xmu_mnu) @ _dag(_roll(U[mu], nu, -1)) @ _roll(U[nu], nu, -1)
    return A


def plaquette(U):
    """Average of Re tr(U_mu(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+) / 3 over n and mu < nu."""
    tot = 0.0
    cnt = 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = U[mu] @ _roll(U[nu], mu, +1) @ _dag(_roll(U[mu], nu, +1)) @ _dag(U[nu])
            tot += np.trace(P, axis1=-2, axis2=-1).real.mean() / 3.0
            cnt += 1
    return tot / cnt


_SUBGROUPS = ((0, 1), (1, 2), (0, 2))


def _kp_sample_x0(rng, alpha):
    """Kennedy-Pendleton: x0 in [-1, 1] with density ~ sqrt(1 - x0^2) exp(alpha x0)."""
    n = alpha.shape[0]
    x0 = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        a = alpha[todo]
        r1 = 1.0 - rng.random(todo.size)
        r2 = rng.random(todo.size)
        r3 = 1.0 - rng.random(todo.size)
        r4 = rng.random(todo.size)
        delta = -(np.log(r1) + np.cos(2.0 * np.pi * r2) ** 2 * np.log(r3)) / a
        ok = r4 * r4 <= 1.0 - 0.5 * delta
        x0[todo[ok]] = 1.0 - delta[ok]
        todo = todo[~ok]
    return x0


def _su2_heatbath(rng, W, i, j, beta):
    """SU(2) subgroup (i, j) update matrices R for links with W = U A (n, 3, 3)."""
    n = W.shape[0]
    w00, w01, w10, w11 = W[:, i, i], W[:, i, j], W[:, j, i], W[:, j, j]
    b0 = 0.5 * (w00 + w11).real
    b3 = 0.5 * (w00 - w11).imag
    b1 = 0.5 * (w01 + w10).imag
    b2 = 0.5 * (w01 - w10).real
    k = np.sqrt(b0 * b0 + b1 * b1 + b2 * b2 + b3 * b3)
    k = np.maximum(k, 1e-300)
    Vm = np.empty((n, 2, 2), dtype=np.complex128)
    Vm[:, 0, 0] = b0 + 1j * b3
    Vm[:, 0, 1] = b2 + 1j * b1
    Vm[:, 1, 0] = -b2 + 1j * b1
    Vm[:, 1, 1] = b0 - 1j * b3
    Vm /= k[:, None, None]
    x0 = _kp_sample_x0(rng, 2.0 * beta * k / 3.0)
    # uniform direction on the sphere for (x1, x2, x3)
    cth = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * np.pi * rng.random(n)
    rad = np.sqrt(np.maximum(1.0 - x0 * x0, 0.0))
    sth = np.sqrt(np.maximum(1.0 - cth * cth, 0.0))
    x1, x2, x3 = rad * sth * np.cos(phi), rad * sth * np.sin(phi), rad * cth
    X = np.empty((n, 2, 2), dtype=np.complex128)
    X[:, 0, 0] = x0 + 1j * x3
    X[:, 0, 1] = x2 + 1j * x1
    X[:, 1, 0] = -x2 + 1j * x1
    X[:, 1, 1] = x0 - 1j * x3
    r = X @ _dag(Vm)
    R = np.zeros((n, 3, 3), dtype=np.complex128)
    R[:, 0, 0] = R[:, 1, 1] = R[:, 2, 2] = 1.0
    R[:, i, i], R[:, i, j], R[:, j, i], R[:, j, j] = r[:, 0, 0], r[:, 0, 1], r[:, 1, 0], r[:, 1, 1]
    return R


def heatbath_gauge(dims, beta=6.0, sweeps=200, seed=0):
    """Wilson-action gauge field after ``sweeps`` Cabibbo-Marinari heatbath sweeps.

    Cold start (all links 1).  One sweep updates, for mu = 0..3 and each site
    parity, every U_mu(n) of that parity by the three SU(2) subgroups in turn
    (links of one direction and parity share no staple).  Reunitarised after
    every sweep.
    """
    rng = np.random.default_rng(seed)
    U = unit_gauge(dims)
    lat = _shape(dims)
    t, z, y, x = np.meshgrid(*[np.arange(L) for L in lat], indexing="ij")
    parity = (t + z + y + x) % 2
    masks = [parity == p for p in (0, 1)]
    for _ in range(sweeps):
        for mu in range(4):
            for p in (0, 1):
                m = masks[p]
                A = staple_sum(U, mu)[m]
                Um = U[mu][m]
                W = Um @ A
                for (i, j) in _SUBGROUPS:
                    R = _su2_heatbath(rng, W, i, j, beta)
                    Um = R @ Um
                    W = R @ W
                U[mu][m] = Um
        U = reunitarize(U)
    return U


# ------------------------------------------------------------------ sources

def gaussian_spinor(dims, seed):
    """Complex Gaussian spinor field, re and im ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    shp = _shape(dims) + (4, 3)
    return rng.standard_normal(shp) + 1j * rng.standard_normal(shp)


def point_source(dims, spin, colour, site=(0, 0, 0, 0)):
    """delta at ``site`` = (x, y, z, t) in one spin-colour component."""
    b = np.zeros(_shape(dims) + (4, 3), dtype=np.complex128)
    x, y, z, t = site
    b[t, z, y, x, spin, colour] = 1.0
    return b
