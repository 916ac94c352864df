"""Write tests/golden/mcrit.json: the critical mass of each seeded beta = 6.0 workload field.

Test infrastructure: calls only the oracle and the seeded input generators.

m_crit is read as minus the smallest real part of the spectrum of the
Wilson-Dirac operator at m = 0 on the given gauge field, so that
D(m_crit + delta) has smallest real eigenvalue part delta (Sec. 1: the
eigenvalues satisfy Re(lambda) > 0 and D turns singular as
Re(lambda_min) -> 0; Sec. 5 quotes m_crit = -0.8049 for its own beta = 6.0,
16^3 x 32 ensemble).  The eigenvalues come from implicitly restarted Arnoldi
(scipy's ARPACK binding, which='SR') on the oracle operator.

Usage: python -m oracle.make_mcrit [--dims 8 8 8 16] [--sweeps 200] [--seed 0] [--threads 8]
       python -m oracle.make_mcrit --field random --dims 4 4 4 4 --seed 0
         (the exp(0.3 i H) field of the small workload instead of a heatbath field)
"""
import argparse
import json
import os
import time

import numpy as np
import scipy.sparse.linalg as sla

from oracle import dirac
from paper_0811_4331_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "..", "tests", "golden", "mcrit.json")


def stencil_matvec(U, threads):
    """D(m = 0) as the oracle's 9-point stencil, applied slab by slab in t on `threads`
    threads (numpy's batched products release the interpreter lock); checked against the
    whole-field operator on a random vector before use."""
    import concurrent.futures
    A = dirac.wilson_stencil(U, 0.0)
    lat = U.shape[1:5]
    T = lat[0]
    n = int(np.prod(lat)) * 12
    bounds = np.linspace(0, T, min(threads, T) + 1).astype(int)
    pool = concurrent.futures.ThreadPoolExecutor(len(bounds) - 1)

    def slab(y, t0, t1, out):
        acc = np.matmul(A[0][t0:t1], y[t0:t1][..., None])[..., 0]
        for d in range(1, 9):
            mu, step = dirac.stencil_offset(d)
            if mu == 3:
                ys = y[(np.arange(t0, t1) + step) % T]
            else:
                ys = np.roll(y[t0:t1], -step, axis=dirac.axis_of(mu))
            acc += np.matmul(A[d][t0:t1], ys[..., None])[..., 0]
        out[t0:t1] = acc

    def mv(v):
        y = v.reshape(lat + (12,))
        out = np.empty_like(y)
        list(pool.map(lambda k: slab(y, bounds[k], bounds[k + 1], out), range(len(bounds) - 1)))
        return out.reshape(n)

    rng = np.random.default_rng(1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = dirac.wilson_dirac(U, x.reshape(lat + (4, 3)), 0.0).reshape(n)
    assert np.linalg.norm(mv(x) - ref) <= 1e-13 * np.linalg.norm(ref)
    return mv


def smallest_real_part(U, nev=4, tol=1e-8, threads=1):
    lat = U.shape[1:5]
    n = int(np.prod(lat)) * 12

    def mv(v):
        return dirac.wilson_dirac(U, v.reshape(lat + (4, 3)), 0.0).reshape(n)

    if threads > 1:
        mv = stencil_matvec(U, threads)

    op = sla.LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    vals = sla.eigs(op, k=nev, which="SR", ncv=64, tol=tol, maxiter=100000,
                    return_eigenvectors=False)
    return float(np.min(vals.real)), [complex(v) for v in vals]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[8, 8, 8, 16])
    ap.add_argument("--beta", type=float, default=6.0)
    ap.add_argument("--sweeps", type=int, default=200)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--field", choices=["heatbath", "random"], default="heatbath")
    ap.add_argument("--threads", type=int, default=1,
                    help="apply the operator as the oracle's stencil on this many threads (t slabs)")
    a = ap.parse_args()
    t0 = time.time()
    if a.field == "random":
        U = inputs.random_gauge(tuple(a.dims), a.seed)
        key = "%dx%dx%dx%d_random0.3_seed%d" % (*a.dims, a.seed)
        how = "python -m oracle.make_mcrit --field random --dims %d %d %d %d --seed %d" % (*a.dims, a.seed)
    else:
        U = inputs.heatbath_gauge(tuple(a.dims), a.beta, a.sweeps, a.seed)
        key = "%dx%dx%dx%d_beta%.1f_sweeps%d_seed%d" % (*a.dims, a.beta, a.sweeps, a.seed)
        how = "python -m oracle.make_mcrit --dims %d %d %d %d --sweeps %d --seed %d" % (*a.dims, a.sweeps, a.seed)
        if a.threads > 1:
            how += " --threads %d" % a.threads
    t1 = time.time()
    lam, vals = smallest_real_part(U, threads=a.threads)
    t2 = time.time()
    data = {}
    if os.path.exists(GOLDEN):
        with open(GOLDEN) as f:
            data = json.load(f)
    data[key] = {
        "dims": a.dims, "field": a.field, "seed": a.seed,
        "plaquette": inputs.plaquette(U),
        "min_re_lambda_m0": lam,
        "m_crit": -lam,
        "lowest_eigenvalues_m0": [[v.real, v.imag] for v in vals],
        "how": how,
        "seconds": {"field": round(t1 - t0, 1), "arnoldi": round(t2 - t1, 1)},
    }
    if a.field == "heatbath":
        data[key].update(beta=a.beta, sweeps=a.sweeps)
    with open(GOLDEN, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print(key, data[key]["m_crit"], data[key]["plaquette"])


if __name__ == "__main__":
    main()
