"""The launch-shape tuner changes speed only.

Every shape of a tuned kernel (threads per CTA of the dslash without fused
dots; right-hand sides per CTA of the tensor-core coarse stencil and
transfers) computes each output with the same instructions in the same
order, so a whole mixed-precision multi-RHS setup + solve gives the same bits
with the default shapes, the first shapes, the last shapes and the tuned ones.
"""
import numpy as np
import pytest

from gpu_util import require_gpu
from paper_0811_4331_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solve(wm, U, dims, B):
    p = wm.mg_default_params(n_levels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 8], setup_sweeps=[6, 6],
                             mixed=1, coarse_mma=1, seed=3)
    h = wm.mg_setup(U, dims, -0.2, p)
    x = np.zeros_like(B)
    _, st = wm.mg_solve(h, B, x, 1e-10)
    wm.mg_destroy(h)
    return x, [s["iters"] for s in st]


def test_every_launch_shape_gives_the_same_bits():
    wm = require_gpu()
    dims = (8, 8, 8, 8)
    U = inputs.random_gauge(dims, 6)
    B = np.stack([inputs.gaussian_spinor(dims, 40 + r) for r in range(12)])
    old = wm.mg_tune(0)
    try:
        x0, it0 = _solve(wm, U, dims, B)
        for mode in (4, 3, 2):
            wm.mg_tune(mode)
            x, it = _solve(wm, U, dims, B)
            assert it == it0, (mode, it, it0)
            assert np.array_equal(x, x0), mode
        rep = wm.mg_tune_report()
        kinds = {k.split("|")[0] for k in rep}
        assert {"dslash", "coarse_mma", "restrict_mma", "prolong_mma"} <= kinds, kinds
        for k, (v, us) in rep.items():
            assert 0 <= v < len(us) and us[v] > 0 and us[v] == min(u for u in us if u > 0), (k, v, us)
    finally:
        wm.mg_tune(old)
