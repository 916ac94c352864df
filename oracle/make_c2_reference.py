"""Write tests/golden/c2_reference.json: the oracle's own MG-GCR solves of the 8^3 x 16 workload.

Test infrastructure: calls only the oracle and the seeded input generators.

Workload: 8^3 x 16 beta = 6.0 heatbath field (200 sweeps, seed 0), masses
m_crit + {0.1, 0.03, 0.01, 0.003}, two levels with 4^4 aggregates, Nv = 20,
300 MR setup sweeps from the counter stream with seed 7, one Gaussian source
(seed 1), GCR(50) to a true relative residual of 1e-10 (Sec. 5 method).
Stored per mass: the outer iteration count, the true residual, and the
solution at a few fixed sites (every component), so that the GPU solution of
the same unique system can be compared site by site.  Under "sweep": the
iteration counts of the mass-sweep form (one setup at the lightest mass, the
same relaxed candidates for every mass, the Galerkin operator per mass).

Usage: python -m oracle.make_c2_reference [--sweep-only]
"""
import json
import os
import time

import numpy as np

from oracle import multigrid as mg
from paper_0811_4331_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "..", "tests", "golden")
DIMS = (8, 8, 8, 16)
DMASSES = (0.1, 0.03, 0.01, 0.003)
SITES = [(0, 0, 0, 0), (7, 7, 7, 15), (3, 5, 1, 9), (6, 0, 4, 12)]


def main():
    sweep_only = "--sweep-only" in os.sys.argv
    with open(os.path.join(GOLDEN, "mcrit.json")) as f:
        mc = json.load(f)["8x8x8x16_beta6.0_sweeps200_seed0"]["m_crit"]
    U = inputs.heatbath_gauge(DIMS, 6.0, 200, 0)
    lat = (DIMS[3], DIMS[2], DIMS[1], DIMS[0])
    b = inputs.gaussian_spinor(DIMS, 1).reshape(lat + (12,))
    starts = [inputs.null_vector_starts(lat, 12, 20, 7)]
    out = {"dims": list(DIMS), "nv": 20, "block": [4, 4, 4, 4], "setup_sweeps": 300, "start_seed": 7,
           "rhs_seed": 1, "tol": 1e-10, "sites_xyzt": SITES, "masses": []}
    if sweep_only:  # keep the per-mass entries, recompute the sweep form only
        with open(os.path.join(GOLDEN, "c2_reference.json")) as f:
            out = json.load(f)
    for dm in (() if sweep_only else DMASSES):
        m = mc + dm
        t0 = time.time()
        h = mg.mg_setup(U, m, [dict(block=(4, 4, 4, 4), nv=20, sweeps=300)], starts)
        t1 = time.time()
        x, info = mg.mg_solve(h, b, tol=1e-10)
        t2 = time.time()
        vals = []
        for (xx, yy, zz, tt) in SITES:
            vals.append([[v.real, v.imag] for v in x[tt, zz, yy, xx]])
        out["masses"].append({"dm": dm, "mass": m, "iters": info["iters"],
                              "true_rel_residual": info["true_rel_residual"],
                              "x_norm": float(np.linalg.norm(x)), "x_at_sites": vals,
                              "seconds": {"setup": round(t1 - t0, 1), "solve": round(t2 - t1, 1)}})
        print(dm, info["iters"], info["true_rel_residual"], t1 - t0, t2 - t1, flush=True)
    # the bench step's form: one setup at the lightest mass, the same candidates at every mass
    # (P from them, A_c = P^+ A(m) P per mass), MG-GCR to the same tolerance
    cands = mg.relax_null_vectors(
        lambda y: __import__("oracle").dirac.wilson_dirac(U, y.reshape(lat + (4, 3)), mc + DMASSES[-1]).reshape(
            lat + (12,)), starts[0], 300)
    out["sweep"] = {"setup_mass": mc + DMASSES[-1], "masses": []}
    for dm in DMASSES:
        m = mc + dm
        h = mg.mg_setup(U, m, [dict(block=(4, 4, 4, 4), nv=20, sweeps=0)], [cands])
        x, info = mg.mg_solve(h, b, tol=1e-10)
        out["sweep"]["masses"].append({"dm": dm, "iters": info["iters"],
                                       "true_rel_residual": info["true_rel_residual"]})
        print("sweep", dm, info["iters"], info["true_rel_residual"], flush=True)
    out["how"] = "python -m oracle.make_c2_reference (single thread)"
    with open(os.path.join(GOLDEN, "c2_reference.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
