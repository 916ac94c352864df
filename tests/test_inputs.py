"""Pins of the seeded input generators (they feed both the CUDA path and the oracle)."""
import os

import numpy as np
import pytest

from paper_0811_4331_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_known_answers():
    lines = [l for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if not l.startswith("#")]
    seed = int(lines[0].split()[1])
    expect = np.array([int(l) for l in lines[1:]], dtype=np.uint64)
    assert np.array_equal(inputs.splitmix64(seed, np.arange(5)), expect)


def test_counter_gaussian_moments_and_offsets():
    g = inputs.counter_gaussian(7, 200000)
    assert abs(g.real.mean()) < 0.01 and abs(g.imag.mean()) < 0.01
    assert abs(g.real.var() - 1) < 0.02 and abs(g.imag.var() - 1) < 0.02
    assert abs(np.mean(g.real * g.imag)) < 0.01
    # counter based: any window is reproducible on its own
    assert np.array_equal(inputs.counter_gaussian(7, 10, offset=1000), g[1000:1010])
    starts = inputs.null_vector_starts((2, 2, 2, 2), 12, 3, 7)
    assert np.array_equal(starts[1].reshape(-1), g[192:384])


def test_random_su3_is_special_unitary():
    U = inputs.random_gauge((4, 4, 2, 2), 0)
    M = U.reshape(-1, 3, 3)
    assert np.max(np.abs(M @ np.conj(np.swapaxes(M, -1, -2)) - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(M) - 1)) < 1e-14


def test_reunitarize_projects_onto_su3():
    rng = np.random.default_rng(0)
    M = inputs.random_su3(rng, 50, 1.0) + 1e-3 * rng.standard_normal((50, 3, 3))
    R = inputs.reunitarize(M)
    assert np.max(np.abs(R @ np.conj(np.swapaxes(R, -1, -2)) - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(R) - 1)) < 1e-14


@pytest.mark.parametrize("beta,lo,hi", [(1.0, 0.045, 0.075),     # strong coupling: beta / 18
                                        (60.0, 0.960, 0.972)])   # weak coupling: 1 - 2 / beta
def test_heatbath_coupling_limits(beta, lo, hi):
    U = inputs.heatbath_gauge((4, 4, 4, 4), beta, 30, seed=1)
    p = inputs.plaquette(U)
    assert lo < p < hi, p


def test_heatbath_beta6_plaquette():
    """beta = 6.0: <P> near the well-known 0.594 (small-volume tolerance)."""
    U = inputs.heatbath_gauge((4, 4, 4, 4), 6.0, 60, seed=2)
    assert 0.585 < inputs.plaquette(U) < 0.605
    M = U.reshape(-1, 3, 3)
    assert np.max(np.abs(np.linalg.det(M) - 1)) < 1e-13


def _digests():
    out = []
    for line in open(os.path.join(GOLDEN, "heatbath_sha256.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out.append((tuple(int(x) for x in f[:4]), float(f[4]), int(f[5]), int(f[6]), f[7]))
    return out


@pytest.mark.parametrize("case", _digests(), ids=lambda c: "x".join(map(str, c[0])))
def test_heatbath_bit_reproducible(case):
    """The heatbath field is identical bit for bit to the stored digest (any machine)."""
    import hashlib
    dims, beta, sweeps, seed, digest = case
    U = inputs.heatbath_gauge(dims, beta, sweeps, seed)
    assert hashlib.sha256(U.tobytes()).hexdigest() == digest
