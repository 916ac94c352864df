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
import ctypes
import os
import subprocess

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


# ------------------------------------------------------------------ heatbath
# The heatbath is plain C (gen/heatbath.c), compiled with -ffp-contract=off
# and restricted to correctly rounded operations, so that the field is the
# same bit for bit on every machine (its critical mass and reference solves
# are stored once).

_GEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gen")
_GEN_LIB = os.path.join(_GEN_DIR, "libgen.so")
_gen = None


def build_generators():
    """Compile gen/heatbath.c into gen/libgen.so (gcc, no FMA contraction)."""
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           os.path.join(_GEN_DIR, "heatbath.c"), "-o", _GEN_LIB + ".tmp", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("building the gauge generator failed:\n" + r.stderr)
    os.replace(_GEN_LIB + ".tmp", _GEN_LIB)
    return _GEN_LIB


def _generators():
    global _gen
    if _gen is None:
        if not os.path.exists(_GEN_LIB):
            build_generators()
        lib = ctypes.CDLL(_GEN_LIB)
        lib.heatbath_su3.restype = ctypes.c_int
        lib.heatbath_su3.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_int,
                                     ctypes.c_uint64]
        _gen = lib
    return _gen


def heatbath_gauge(dims, beta=6.0, sweeps=200, seed=0):
    """Wilson-action gauge field after ``sweeps`` Cabibbo-Marinari heatbath sweeps (cold start).

    Three SU(2) subgroups per link, each by Kennedy-Pendleton; mu = 0..3, even
    then odd sites per sweep; reunitarised after every sweep; random numbers
    from one SplitMix64 stream seeded with ``seed``.  See gen/heatbath.c.
    """
    lat = _shape(dims)
    U = np.empty((4,) + lat + (3, 3), dtype=np.complex128)
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    _generators().heatbath_su3(U.ctypes.data, d, float(beta), int(sweeps), int(seed))
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
