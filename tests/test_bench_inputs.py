"""The 32^3 x 64 workload's field is the 16^3 x 32 field tiled 2 x 2 x 2 x 2 (bench.tile_gauge).  A tiled
periodic field is again SU(3) with the same plaquette, and the Wilson operator commutes with tiling:
D_big (tile psi) = tile (D_small psi), so the small lattice's spectrum (and critical mass) is part of the
big one's.  Checked on CPU with the oracle operator on small lattices and uneven tilings."""
import os
import sys

import numpy as np

from oracle import dirac
from paper_0811_4331_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tile_field(psi, reps):
    out = psi
    for ax, r in zip(range(0, 4), reversed(reps)):  # psi axes (Lt, Lz, Ly, Lx, 4, 3)
        out = np.concatenate([out] * r, axis=ax)
    return out


def test_tiling_commutes_with_the_operator():
    sys.path.insert(0, ROOT)
    import bench
    dims = (2, 3, 2, 2)
    reps = (2, 1, 3, 2)
    U = inputs.random_gauge(dims, 4)
    Ub = bench.tile_gauge(U, reps)
    assert Ub.shape[1:5] == (4, 6, 3, 4)
    flat = Ub.reshape(-1, 3, 3)
    assert np.max(np.abs(flat @ np.conj(np.swapaxes(flat, -1, -2)) - np.eye(3))) < 1e-13
    assert np.max(np.abs(np.linalg.det(flat) - 1.0)) < 1e-13
    assert abs(inputs.plaquette(Ub) - inputs.plaquette(U)) < 1e-13
    psi = inputs.gaussian_spinor(dims, 5)
    m = -0.3
    lhs = dirac.wilson_dirac(Ub, _tile_field(psi, reps), m)
    rhs = _tile_field(dirac.wilson_dirac(U, psi, m), reps)
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.max(np.abs(rhs))
