"""Qualitative pin of the paper's claim (Secs. 4-5): multigrid removes critical slowing down.

As the mass approaches its critical value the unpreconditioned Krylov solver's iteration count grows
(the Wilson operator's smallest eigenvalue shrinks with m - m_crit), while MG-GCR, whose prolongator
holds the near-null space, keeps a nearly constant count.  The paper prints no numbers, so iteration
counts are otherwise unpinned; this checks the shape of its comparison on the oracle.

Field: the small workload's exp(0.3 i H) field on 4^4 (seed 0), m_crit = -(smallest Re lambda of D at
m = 0) from tests/golden/mcrit.json (written by oracle/make_mcrit.py with ARPACK on the oracle operator).
MG: 2^4 blocks, Nv = 12 null vectors from 50 MR relaxation sweeps each (Sec. 2), V(2,2), exact coarsest
solve, GCR(50), tol 1e-10.
"""
import json
import os

import numpy as np

from oracle import dirac, krylov
from oracle import multigrid as mg
from paper_0811_4331_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mcrit.json")


def test_mg_iterations_stay_flat_while_bicgstab_grows():
    dims = (4, 4, 4, 4)
    lat = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 0)
    with open(GOLDEN) as f:
        mc = json.load(f)["4x4x4x4_random0.3_seed0"]["m_crit"]
    b = inputs.gaussian_spinor(dims, 1)
    starts = [inputs.gaussian_spinor(dims, 100 + k).reshape(lat + (12,)) for k in range(12)]
    spec = dict(block=(2, 2, 2, 2), nv=12, sweeps=50)
    bicg, mgit = {}, {}
    for dm in (0.3, 0.03, 0.01):
        m = mc + dm
        _, info = krylov.bicgstab(lambda v: dirac.wilson_dirac(U, v, m), b, 1e-10)
        bicg[dm] = info["iters"]
        hier = mg.mg_setup(U, m, [spec], [starts])
        x, inf2 = mg.mg_solve(hier, b.reshape(lat + (12,)), tol=1e-10)
        assert np.linalg.norm(b.reshape(x.shape) - hier[0].apply(x)) <= 1.01e-10 * np.linalg.norm(b)
        mgit[dm] = inf2["iters"]
    assert bicg[0.01] >= 3 * bicg[0.3], bicg              # Krylov slows down towards m_crit
    assert mgit[0.01] <= 1.25 * mgit[0.3] + 1, mgit       # multigrid does not
    assert mgit[0.01] * 10 < bicg[0.01], (mgit, bicg)
