"""GPU parity of the multigrid setup and transfer pieces against the oracle.

Same seeded inputs on both sides (gauge field, start vectors).  Tolerances:
P and the coarse stencil 1e-10 (FP64; the relaxation and Gram-Schmidt
rounding of two implementations differs at 1e-16 per operation and is
amplified by the conditioning of each aggregate's candidate block),
restriction / prolongation / coarse apply 1e-12 given the same P, one
V-cycle 1e-9.
"""
import numpy as np
import pytest

from gpu_util import lattice, rel_err, require_gpu, torch
from oracle import dirac
from oracle import multigrid as mg
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle_vectors(P, nv, nhalf):
    """Oracle P (lattice + (ncomp, 2 nv)) -> nv vectors (lattice + (ncomp,)) as the library exports them."""
    v = np.concatenate([P[..., :nhalf, :nv], P[..., nhalf:, nv:]], axis=-2)
    return np.moveaxis(v, -1, 0)


def _setup_both(wm, dims, mass, levels, seed=0, device_starts=False, pseed=7, adapt=(0, 3)):
    U = inputs.random_gauge(dims, seed)
    lat = lattice(dims)
    starts, shapes = [], [(lat, 12)]
    for spec in levels:
        shp, nc = shapes[-1]
        starts.append(inputs.null_vector_starts(shp, nc, spec["nv"], pseed + len(starts)))
        blk = mg.Blocking(shp, spec["block"], nc)
        shapes.append((blk.coarse, 2 * spec["nv"]))
    p = wm.mg_default_params(n_levels=len(levels) + 1, block=[s["block"] for s in levels],
                             nv=[s["nv"] for s in levels], setup_sweeps=[s["sweeps"] for s in levels],
                             seed=pseed, adapt_steps=adapt[0], adapt_cycles=adapt[1],
                             adapt_nv=[s.get("adapt_nv", 0) for s in levels])
    h = wm.mg_setup(U, dims, mass, p, starts=None if device_starts else
                    [np.stack(s).reshape(len(s), -1, s[0].shape[-1]) for s in starts])
    levels_o = [dict(sp, adapt_steps=adapt[0], adapt_cycles=adapt[1]) for sp in levels]
    hier = mg.mg_setup(U, mass, levels_o, starts, coarse_cycles=(p.coarse_cycles[0],))
    return h, hier, U


CASES = [
    ((4, 4, 4, 4), [dict(block=(2, 2, 2, 2), nv=8, sweeps=10)]),        # the small 4^4 workload
    ((6, 4, 2, 4), [dict(block=(2, 2, 2, 2), nv=5, sweeps=3)]),         # coarse extents 3, 2, 1, 2
    ((4, 4, 4, 4), [dict(block=(2, 2, 2, 2), nv=4, sweeps=4),            # three levels
                    dict(block=(2, 2, 1, 1), nv=3, sweeps=4)]),
]


@pytest.mark.parametrize("dims,levels", CASES)
def test_prolongator_and_coarse_operator(dims, levels):
    wm = require_gpu()
    h, hier, U = _setup_both(wm, dims, 0.1, levels)
    for l, spec in enumerate(levels):
        got = wm.mg_get_prolongator(h, l)
        nhalf = hier[l].ncomp // 2
        want = _oracle_vectors(hier[l].P, spec["nv"], nhalf).reshape(got.shape)
        assert np.max(np.abs(got - want)) < 1e-10, (l, np.max(np.abs(got - want)))
        Ac = wm.mg_get_coarse_op(h, l + 1)
        want_c = hier[l + 1].stencil.reshape(Ac.shape)
        assert np.max(np.abs(Ac - want_c)) < 1e-10 * np.max(np.abs(want_c)), l


# (dims, levels, solver iterations per prototype).  The second level of the 3-level
# case has 160 unknowns: more iterations there would solve A x = 0 to rounding
# level, leaving a prototype made of rounding noise on either side.
ADAPT_CASES = [
    ((4, 4, 4, 4), [dict(block=(2, 2, 2, 2), nv=8, sweeps=6, adapt_nv=5)], 10),   # batches of 3 and 2; a restart
    ((4, 4, 4, 4), [dict(block=(2, 2, 2, 2), nv=5, sweeps=4, adapt_nv=2),        # three levels, both adaptive
                    dict(block=(2, 2, 1, 1), nv=4, sweeps=4, adapt_nv=2)], 3),
]


@pytest.mark.parametrize("device_starts", [False, True])
@pytest.mark.parametrize("dims,levels,iters", ADAPT_CASES)
def test_adaptive_setup_matches_oracle(dims, levels, iters, device_starts):
    """Adaptive steps (Sec. 2: V^k augmented by prototypes from the current solver
    applied to A x = 0), two steps per level: P and the coarse operators of every
    level match the oracle's.  The prototypes pass through whole V-cycles, so the
    tolerance is the V-cycle's (1e-9) amplified by the block QR's conditioning: 1e-8."""
    wm = require_gpu()
    h, hier, U = _setup_both(wm, dims, 0.1, levels, adapt=(2, iters), device_starts=device_starts)
    for l, spec in enumerate(levels):
        got = wm.mg_get_prolongator(h, l)
        nhalf = hier[l].ncomp // 2
        want = _oracle_vectors(hier[l].P, spec["nv"], nhalf).reshape(got.shape)
        assert np.max(np.abs(got - want)) < 1e-8, (l, np.max(np.abs(got - want)))
        Ac = wm.mg_get_coarse_op(h, l + 1)
        want_c = hier[l + 1].stencil.reshape(Ac.shape)
        assert np.max(np.abs(Ac - want_c)) < 1e-8 * np.max(np.abs(want_c)), l


def test_adaptive_setup_mixed_solves():
    """The mixed hierarchy (FP32 relaxation, FP32 GCR with the 16-bit V-cycle making the prototypes)
    with half of its Nv = 12 vectors from two adaptive steps gives a solve to the
    1e-10 true FP64 residual."""
    wm = require_gpu()
    dims = (8, 8, 8, 8)
    U = inputs.random_gauge(dims, 2)
    b = inputs.gaussian_spinor(dims, 3)
    p = wm.mg_default_params(mixed=1, nv=[12], setup_sweeps=[10], adapt_steps=2, adapt_nv=[6])
    h = wm.mg_setup(U, dims, -0.2, p)
    x = np.zeros_like(b)
    wm.mg_solve(h, b, x, 1e-10)
    r = b.reshape(lattice(dims) + (4, 3)) - dirac.wilson_dirac(U, x.reshape(lattice(dims) + (4, 3)), -0.2)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b) * 1.01


def test_device_start_vectors_follow_the_counter_definition():
    """starts=None: the on-device SplitMix64/Box-Muller starts equal inputs.null_vector_starts."""
    wm = require_gpu()
    dims = (4, 4, 4, 4)
    levels = [dict(block=(2, 2, 2, 2), nv=6, sweeps=2)]
    h, hier, U = _setup_both(wm, dims, 0.1, levels, device_starts=True, pseed=123)
    got = wm.mg_get_prolongator(h, 0)
    want = _oracle_vectors(hier[0].P, 6, 6).reshape(got.shape)
    assert np.max(np.abs(got - want)) < 1e-10


def test_rank_loss_is_reported():
    wm = require_gpu()
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 0)
    v = inputs.null_vector_starts(lattice(dims), 12, 1, 5)[0]
    starts = [np.stack([v, (0.5 - 1j) * v]).reshape(2, -1, 12)]
    p = wm.mg_default_params(n_levels=2, block=[(2, 2, 2, 2)], nv=[2], setup_sweeps=[0])
    with pytest.raises(wm.MgError) as e:
        wm.mg_setup(U, dims, 0.1, p, starts=starts)
    assert e.value.status == wm.MG_ERANK




def test_non_su3_gauge_field_is_refused():
    """The mixed operators rebuild each link's third row as for SU(3), so mg_setup checks every link."""
    wm = require_gpu()
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 0)
    p = wm.mg_default_params(n_levels=1, mixed=1)
    wm.mg_destroy(wm.mg_setup(U, dims, 0.1, p))  # SU(3) to rounding: accepted
    bad = U.copy()
    bad[2, 1, 3, 0, 2] *= 1.0 + 1e-6  # one link (mu = z, t = 1, z = 3, y = 0, x = 2) off by 1e-6
    with pytest.raises(wm.MgError) as e:
        wm.mg_setup(bad, dims, 0.1, p)
    assert e.value.status == wm.MG_EINVAL and "SU(3)" in str(e.value)
    phase = U.copy()
    phase[0, 0, 0, 0, 1] *= np.exp(0.5j)  # unitary, det != 1
    with pytest.raises(wm.MgError):
        wm.mg_setup(phase, dims, 0.1, p)

def test_block_too_large_for_the_galerkin_tile_is_refused():
    """A block whose P column does not fit the Galerkin CTA's shared memory is refused with a message."""
    wm = require_gpu()
    dims = (8, 8, 8, 8)
    U = inputs.random_gauge(dims, 0)
    for mixed, ok in ((0, (4, 4, 4, 8)), (1, (4, 4, 8, 8))):  # 512 sites FP64, 1024 sites FP32 still fit
        p = wm.mg_default_params(n_levels=2, block=[(8, 8, 8, 8)], nv=[4], setup_sweeps=[0], mixed=mixed)
        with pytest.raises(wm.MgError) as e:
            wm.mg_setup(U, dims, 0.1, p)
        assert e.value.status == wm.MG_EINVAL and "shared memory" in str(e.value), str(e.value)
        p = wm.mg_default_params(n_levels=2, block=[ok], nv=[4], setup_sweeps=[0], mixed=mixed)
        wm.mg_destroy(wm.mg_setup(U, dims, 0.1, p))

def _to_dev(wm, h, level, arr, prec=0, nrhs=1):
    t = wm.internal_empty(h, level, prec, nrhs)
    wm.mg_field_to_internal(h, level, prec, torch.from_numpy(np.ascontiguousarray(arr)).cuda(), t, nrhs)
    return t


def _to_host(wm, h, level, t, shape, prec=0, nrhs=1):
    e = torch.empty(shape, dtype=torch.complex128, device="cuda")
    wm.mg_field_from_internal(h, level, prec, t, e, nrhs)
    return e.cpu().numpy()


def test_transfer_coarse_apply_mr_and_vcycle():
    wm = require_gpu()
    dims = (4, 4, 4, 4)
    levels = [dict(block=(2, 2, 2, 2), nv=6, sweeps=5), dict(block=(2, 2, 1, 1), nv=3, sweeps=5)]
    h, hier, U = _setup_both(wm, dims, -0.2, levels)
    lat = lattice(dims)
    blk = hier[0].blk
    rng = np.random.default_rng(4)
    r = rng.standard_normal(lat + (12,)) + 1j * rng.standard_normal(lat + (12,))
    rc = rng.standard_normal(blk.coarse + (12,)) + 1j * rng.standard_normal(blk.coarse + (12,))
    # restriction / prolongation with the library's P, against the oracle with the oracle's P
    rd = _to_dev(wm, h, 0, r)
    out = wm.internal_empty(h, 1, 0)
    wm.restrict_apply(h, 0, 0, rd, out)
    assert rel_err(_to_host(wm, h, 1, out, rc.shape), mg.restrict(hier[0].P, blk, r)) < 1e-10
    cd = _to_dev(wm, h, 1, rc)
    fo = wm.internal_empty(h, 0, 0)
    wm.prolong_apply(h, 0, 0, cd, fo)
    assert rel_err(_to_host(wm, h, 0, fo, r.shape), mg.prolong(hier[0].P, blk, rc)) < 1e-10
    # coarse stencil apply
    co = wm.internal_empty(h, 1, 0)
    wm.coarse_apply(h, 1, 0, cd, co)
    assert rel_err(_to_host(wm, h, 1, co, rc.shape), dirac.stencil_apply(hier[1].stencil, rc)) < 1e-10
    # MR on the coarse level
    xd = _to_dev(wm, h, 1, np.zeros_like(rc))
    resd = wm.internal_empty(h, 1, 0)
    wm.mr_apply(h, 1, 0, cd, xd, resd, 4)
    xo, _ = mg.mr_relax(hier[1].apply, rc, np.zeros_like(rc), 4, 0.8)
    assert rel_err(_to_host(wm, h, 1, xd, rc.shape), xo) < 1e-9
    # one modified V-cycle (3 levels: 4 level-1 V-cycles per fine coarse correction)
    ed = wm.internal_empty(h, 0, 0)
    wm.vcycle_apply(h, rd, ed)
    eo = mg.vcycle(hier, 0, r, 2, 2, 0.8, (4,))
    assert rel_err(_to_host(wm, h, 0, ed, r.shape), eo) < 1e-9
