"""Oracle: adaptive multigrid for the Wilson-Dirac system, plain FP64 (test infrastructure only).

Every function follows a passage of the paper (Clark et al., Lattice 2008):

* ``mr_relax``            -- the under-relaxed minimal-residual smoother with
                             omega = 0.8 (Sec. 3, last paragraph).
* ``relax_null_vectors``  -- adaptive steps 1-2 of Sec. 2: relax A x = 0 from a
                             random x0 for l iterations; the iterate is a
                             candidate v.
* ``block_orthonormalize``-- Sec. 2 step 3 and Eq. (2.3): split the candidates
                             over aggregates and QR them, P V_c = V, P^+ P = 1;
                             the split also keeps chirality, [gamma5, P] = 0
                             (Sec. 3 after Eq. 3.2; Sec. 5: like chirality in
                             a block).
* ``restrict``/``prolong``-- R = P^+ and P (Sec. 3, Eq. 3.2 and the text after).
* ``coarse_stencil``      -- the Galerkin coarse operator A_c = P^+ A P (Sec. 2),
                             written as a 9-point stencil of coarse blocks.
* ``vcycle``              -- V(2,2) (Sec. 2) with the coarse-grid correction
                             damped by alpha = <A x_c|r0>/<A x_c|A x_c>
                             (Sec. 3, Eq. 3.5) and the modified cycle of Sec. 5:
                             4 applications of the next level's V-cycle
                             between restriction and prolongation on the fine
                             grid.
* ``build_levels``        -- the adaptive steps of Sec. 2 beyond relaxation:
                             the current solver (MG-preconditioned GCR)
                             applied to A x = 0 from a random start gives the
                             next prototype, appended to V^k, P rebuilt.
* ``fgcr``                -- GCR(50) as the outer Krylov method (Sec. 5),
                             flexible because the preconditioner varies.

Not in the paper: ``mg_setup(..., fine_smoother="eo")`` replaces the fine
level's MR smoother by the even-odd one of ``evenodd.eo_smooth`` (MR on the
Schur complement, odd sites solved exactly) in every cycle, including those
the adaptive steps run.

Readings where the paper is silent: one relaxation =
one MR step; candidates start from independent Gaussian vectors, get l MR
steps on A x = 0 with omega = 0.8 and are normalised to unit norm; the QR is
modified Gram-Schmidt applied twice, in candidate order; the chirality split
of a level with ncomp components per site puts components [0, ncomp/2) in
chirality + and [ncomp/2, ncomp) in chirality -; the same smoother and alpha
step are used on every level; the coarsest level is solved exactly by dense
LU; the 4 coarse applications are 4 steps of flexible GCR on the coarse
equation preconditioned by the next level's V-cycle, from e_c = 0 (4
stationary sweeps e_c += V(r_c - A_c e_c) are the alternative reading,
``coarse_solver="stationary"``); an adaptive step runs a fixed number of
iterations of flexible GCR preconditioned by the level's V-cycle (restarted
every 8) from a random start and appends a batch of such vectors at once
(each batch made with the solver of the V^k before it); the levels below are
rebuilt from scratch after each step; inner products are <a|b> = sum conj(a) b.

Field arrays have shape (Lt, Lz, Ly, Lx, ncomp); a block size is given as
(bx, by, bz, bt), matching the x-fastest site order.
"""
import numpy as np
import scipy.linalg

from . import dirac


def inner(a, b):
    """<a|b> = sum conj(a) b."""
    return np.vdot(a, b)


def norm2(a):
    return float(np.vdot(a, a).real)


# ---------------------------------------------------------------- smoother

def minimal_residual_coefficient(p, r):
    """alpha = <p|r>/<p|p>, the minimiser of ||r - alpha p|| (Sec. 3, Eq. 3.5 with p = D x_c).

    Returns 0 when p = 0.
    """
    pp = norm2(p)
    if pp == 0.0:
        return 0.0
    return inner(p, r) / pp


def mr_relax(apply, b, x, steps, omega=0.8):
    """Under-relaxed minimal residual on A x = b (Sec. 3).

    Each step takes p = A r, alpha = <p|r>/<p|p> (the minimiser of
    ||r - alpha p||) and moves x by omega alpha r.  ``x=None`` means a zero
    initial guess (no operator application is spent on it).  A step with
    <p|p> = 0 leaves x and r unchanged.  Returns (x, r) with r the updated
    residual b - A x.
    """
    if x is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x.copy()
        r = b - apply(x)
    for _ in range(steps):
        p = apply(r)
        alpha = minimal_residual_coefficient(p, r)
        x = x + omega * alpha * r
        r = r - omega * alpha * p
    return x, r


def relax_null_vectors(apply, starts, sweeps, omega=0.8):
    """Candidates for the near null space (Sec. 2, adaptive steps 1-2).

    For each random start x0: ``sweeps`` MR steps on A x = 0, then the iterate
    is normalised to unit 2-norm.
    """
    out = []
    for x0 in starts:
        x, _ = mr_relax(apply, np.zeros_like(x0), x0, sweeps, omega)
        out.append(x / np.sqrt(norm2(x)))
    return out


# ---------------------------------------------------------------- aggregates

class Blocking:
    """Regular geometric aggregates (Sec. 3, first paragraph) plus the chirality split."""

    def __init__(self, lattice, block, ncomp):
        # lattice: numpy shape (Lt, Lz, Ly, Lx); block: (bx, by, bz, bt)
        self.lattice = tuple(lattice)
        self.block = tuple(block)
        self.bnp = tuple(reversed(block))  # (bt, bz, by, bx)
        for L, b in zip(self.lattice, self.bnp):
            if L % b:
                raise ValueError("lattice not divisible by block")
        self.coarse = tuple(L // b for L, b in zip(self.lattice, self.bnp))
        self.ncomp = ncomp
        self.half = ncomp // 2

    def chirality(self, c):
        return 0 if c < self.half else 1

    def block_sum(self, f):
        """Sum a fine-site array (lattice + tail) over each aggregate."""
        tail = f.shape[4:]
        shp = []
        for C, b in zip(self.coarse, self.bnp):
            shp += [C, b]
        g = f.reshape(tuple(shp) + tail)
        return g.sum(axis=(1, 3, 5, 7))

    def broadcast(self, fc):
        """Copy a coarse-site array onto every fine site of its aggregate."""
        g = fc
        for ax, b in enumerate(self.bnp):
            g = np.repeat(g, b, axis=ax)
        return g

    def coords(self, mu):
        """Coordinate n_mu of every fine site, shape = lattice."""
        ax = dirac.axis_of(mu)
        shape = [1, 1, 1, 1]
        shape[ax] = self.lattice[ax]
        c = np.arange(self.lattice[ax]).reshape(shape)
        return np.broadcast_to(c, self.lattice)


def mgs2(Vb):
    """Modified Gram-Schmidt, two passes, columns in order (Sec. 2, Eq. 2.3: the Q of a QR).

    Raises ArithmeticError on rank loss (a column shrinks below 1e-12 of its
    original norm).
    """
    n, k = Vb.shape
    Q = np.zeros((n, k), dtype=np.complex128)
    for i in range(k):
        q = Vb[:, i].copy()
        orig = np.sqrt(norm2(q))
        for _ in range(2):
            for j in range(i):
                q = q - inner(Q[:, j], q) * Q[:, j]
        nq = np.sqrt(norm2(q))
        if not nq > 1e-12 * orig:
            raise ArithmeticError("block Gram-Schmidt: rank loss")
        Q[:, i] = q / nq
    return Q


def block_orthonormalize(cands, blk):
    """P from the candidates (Sec. 2 step 3 and Eq. 2.3; chirality kept, Sec. 3).

    Returns P with shape lattice + (ncomp, 2 Nv): P(n)[c, chi * Nv + k] is
    column k of the Q factor of aggregate B(n), chirality chi = chirality(c);
    entries with chirality(c) != chi are structurally zero.
    """
    nv = len(cands)
    V = np.stack(cands, axis=-1)  # lattice + (ncomp, Nv)
    P = np.zeros(blk.lattice + (blk.ncomp, 2 * nv), dtype=np.complex128)
    shp = []
    for C, b in zip(blk.coarse, blk.bnp):
        shp += [C, b]
    Vr = V.reshape(tuple(shp) + (blk.ncomp, nv))
    Pr = P.reshape(tuple(shp) + (blk.ncomp, 2 * nv))
    h = blk.half
    for B in np.ndindex(*blk.coarse):
        sl = (B[0], slice(None), B[1], slice(None), B[2], slice(None), B[3], slice(None))
        for chi in range(2):
            comps = slice(chi * h, (chi + 1) * h)
            piece = Vr[sl][..., comps, :]  # (bt, bz, by, bx, h, Nv)
            Q = mgs2(piece.reshape(-1, nv))
            Pr[sl][..., comps, chi * nv:(chi + 1) * nv] = Q.reshape(piece.shape)
    return P


def restrict(P, blk, r):
    """r_c(B) = sum_{n in B} P(n)^+ r(n)  (R = P^+, Sec. 3)."""
    return blk.block_sum(np.einsum("...ci,...c->...i", np.conj(P), r))


def prolong(P, blk, xc):
    """x(n) = P(n) x_c(B(n))  (Sec. 2)."""
    return np.einsum("...ci,...i->...c", P, blk.broadcast(xc))


def coarse_stencil(A, P, blk):
    """A_c = P^+ A P (Sec. 2) as a 9-point stencil on the coarse lattice.

    C_{d'}(B) = sum over fine sites n in B and fine hops d whose target n + e_d
    lies in the aggregate reached from B by coarse hop d' of
    P(n)^+ A_d(n) P(n + e_d).  A hop +mu leaves its aggregate when
    n_mu mod b_mu = b_mu - 1, a hop -mu when n_mu mod b_mu = 0; every other
    hop stays in B (d' = 0).  The +mu and -mu blocks are kept apart even when
    the coarse extent is 1 or 2 and both reach the same coarse site.
    """
    nc = P.shape[-1]
    Ac = np.zeros((9,) + blk.coarse + (nc, nc), dtype=np.complex128)
    Pc = np.conj(P)
    for d in range(9):
        if d == 0:
            M = np.einsum("...ci,...cd,...dj->...ij", Pc, A[0], P, optimize=True)
            Ac[0] += blk.block_sum(M)
            continue
        mu, step = dirac.stencil_offset(d)
        M = np.einsum("...ci,...cd,...dj->...ij", Pc, A[d], dirac.shift(P, mu, step), optimize=True)
        b = blk.block[mu]
        n = blk.coords(mu) % b
        leaves = (n == b - 1) if step > 0 else (n == 0)
        leaves = leaves[..., None, None]
        Ac[d] += blk.block_sum(np.where(leaves, M, 0))
        Ac[0] += blk.block_sum(np.where(leaves, 0, M))
    return Ac


def dense_from_stencil(A):
    """Dense matrix of a stencil operator (brute-force helper for tests)."""
    lat = A.shape[1:5]
    nc = A.shape[-1]
    return dirac.dense_matrix(lambda y: dirac.stencil_apply(A, y), lat + (nc,))


# ---------------------------------------------------------------- hierarchy

class Level:
    def __init__(self, apply, lattice, ncomp):
        self.apply = apply
        self.lattice = tuple(lattice)
        self.ncomp = ncomp
        self.P = None
        self.blk = None
        self.stencil = None
        self.lu = None
        self.smooth = None  # (r, steps, omega) -> (e, r - A e); None = MR on A


def smooth(lev, r, steps, omega):
    """The level's smoother from e = 0: MR on A (Sec. 3) unless the level carries another."""
    if lev.smooth is not None:
        return lev.smooth(r, steps, omega)
    return mr_relax(lev.apply, r, None, steps, omega)


def mg_setup(U, mass, levels, starts, omega=0.8, nu_pre=2, nu_post=2, coarse_cycles=(4,), coarse_solver="gcr",
             fine_smoother="mr"):
    """Build the multigrid hierarchy (Sec. 2 adaptive steps, Sec. 3, Sec. 5).

    ``levels`` lists, for every level that gets a coarser one below it, a dict
    with ``block`` (bx, by, bz, bt), ``nv`` and ``sweeps``, and optionally
    ``adapt_nv``, ``adapt_steps`` and ``adapt_cycles`` (see ``build_levels``).
    ``starts[l]`` are the Nv random start vectors of level l (arrays shaped
    like that level's fields).  The coarsest level gets a dense LU
    factorisation.  The cycle options are those the adaptive steps run;
    ``fine_smoother`` is "mr" (Sec. 3) or "eo" (even-odd, module header).
    """
    lat = U.shape[1:5]
    fine = Level(None, lat, 12)
    fine.stencil = dirac.wilson_stencil(U, mass)

    def apply_fine(y):
        return dirac.wilson_dirac(U, y.reshape(lat + (4, 3)), mass).reshape(lat + (12,))

    fine.apply = apply_fine
    if fine_smoother == "eo":  # even-odd smoother on the fine level (not in the paper)
        from .evenodd import eo_smooth

        def smooth_eo(r, steps, om):
            e, res = eo_smooth(U, mass, r.reshape(lat + (4, 3)), steps, om)
            return e.reshape(lat + (12,)), res.reshape(lat + (12,))

        fine.smooth = smooth_eo
    hier = [fine]
    cycle = dict(nu_pre=nu_pre, nu_post=nu_post, omega=omega, coarse_cycles=coarse_cycles,
                 coarse_solver=coarse_solver)
    build_levels(hier, 0, levels, starts, omega, cycle)
    return hier


def coarsen(hier, l, cands, spec):
    """P of level l from the candidates (Eq. 2.3) and A_{l+1} = P^+ A_l P (Sec. 2);
    replaces every level below l."""
    cur = hier[l]
    del hier[l + 1:]
    blk = Blocking(cur.lattice, spec["block"], cur.ncomp)
    cur.blk = blk
    cur.P = block_orthonormalize(cands, blk)
    Ac = coarse_stencil(cur.stencil, cur.P, blk)
    nxt = Level(None, blk.coarse, 2 * len(cands))
    nxt.stencil = Ac
    nxt.apply = (lambda A: (lambda y: dirac.stencil_apply(A, y)))(Ac)
    hier.append(nxt)


def adaptive_prototype(hier, l, x, iters, cycle, restart=8):
    """The current solver of level l -- flexible GCR preconditioned by the level's
    multigrid cycle (Sec. 5) -- applied to A x = 0 from x for ``iters``
    iterations, restarted every ``restart`` (Sec. 2: its iterate is the next
    prototype of the algebraically smooth error)."""
    A = hier[l].apply

    def precond(v):
        return vcycle(hier, l, v, **cycle)

    done = 0
    while done < iters:
        k = min(restart, iters - done)
        x = x + gcr_fixed(A, -A(x), precond, k)
        done += k
    return x


def build_levels(hier, l, levels, starts, omega, cycle):
    """Levels l+1 .. coarsest below the operator of level l (Sec. 2).

    V^k of level l starts with the first Nv - adapt_nv candidates from
    relaxation (``relax_null_vectors``).  It is then augmented in
    ``adapt_steps`` batches -- batch s holds adapt_nv // steps vectors, one
    more for s < adapt_nv % steps -- each vector the result of ``adapt_cycles``
    iterations of the current solver on A x = 0 from its random start
    (``adaptive_prototype``), unit-normalised (Sec. 2: the current solver
    applied to A x = 0 gives the next prototype).  After every change of V^k the prolongator is
    rebuilt and the levels below are built again by this same procedure.
    ``starts[l]`` are always shaped for the final hierarchy; a level built
    while the level above has k < Nv candidates takes, of each start, the
    first k components of each chirality half.
    """
    if l == len(levels):
        hier[l].lu = scipy.linalg.lu_factor(dense_from_stencil(hier[l].stencil))
        return
    spec = levels[l]
    cur = hier[l]
    nv = spec["nv"]
    steps = spec.get("adapt_steps", 0)
    na = spec.get("adapt_nv", 0) if steps > 0 else 0
    if not 0 <= na < nv:
        raise ValueError("adapt_nv must be in [0, nv)")
    steps = min(steps, na)
    k0 = nv - na
    st = starts[l]
    if st[0].shape[-1] > cur.ncomp:
        # while the level above is still short of its Nv candidates this level
        # has fewer components: its starts are the full-size ones restricted to
        # the components that exist (the first k of each chirality half)
        k, kf = cur.ncomp // 2, st[0].shape[-1] // 2
        comps = list(range(k)) + list(range(kf, kf + k))
        st = [v[..., comps] for v in st]
    cands = relax_null_vectors(cur.apply, st[:k0], spec["sweeps"], omega)
    coarsen(hier, l, cands, spec)
    build_levels(hier, l + 1, levels, starts, omega, cycle)
    nxt = k0
    for s in range(steps):
        q = na // steps + (1 if s < na % steps else 0)
        for x in st[nxt:nxt + q]:
            x = adaptive_prototype(hier, l, x, spec.get("adapt_cycles", 16), cycle)
            cands.append(x / np.sqrt(norm2(x)))
        nxt += q
        coarsen(hier, l, cands, spec)
        build_levels(hier, l + 1, levels, starts, omega, cycle)


def coarsest_solve(level, r):
    """Exact solve on the coarsest level by dense LU."""
    return scipy.linalg.lu_solve(level.lu, r.reshape(-1)).reshape(r.shape)


def gcr_fixed(apply, b, precond, iters):
    """``iters`` steps of flexible GCR on A x = b from x = 0 (modified Gram-Schmidt, no
    restart, no stopping test): the Krylov-accelerated form of applying a preconditioner
    ``iters`` times."""
    x = np.zeros_like(b)
    r = b.copy()
    Z, W = [], []
    for _ in range(iters):
        z = precond(r)
        w = apply(z)
        for j in range(len(W)):
            beta = inner(W[j], w)
            w = w - beta * W[j]
            z = z - beta * Z[j]
        nw = np.sqrt(norm2(w))
        if nw == 0.0:
            break
        w = w / nw
        z = z / nw
        a = inner(w, r)
        x = x + a * z
        r = r - a * w
        Z.append(z)
        W.append(w)
    return x


def vcycle(hier, l, r, nu_pre=2, nu_post=2, omega=0.8, coarse_cycles=(4,), coarse_solver="gcr"):
    """One modified V(nu_pre, nu_post) cycle on level l applied to residual r.

    Pre-smooth from e = 0, restrict, solve the coarse equation (exactly on the
    coarsest level, else by ``coarse_cycles[l]`` applications of the next
    level's V-cycle: as flexible GCR steps preconditioned by it, the default,
    or as stationary sweeps e_c += V(r_c - A_c e_c)), prolong to x_c, add
    alpha x_c with alpha = <A x_c|r0>/<A x_c|A x_c> (Eq. 3.5), post-smooth.
    """
    lev = hier[l]
    if l == len(hier) - 1:
        return coarsest_solve(lev, r)
    e, res = smooth(lev, r, nu_pre, omega)
    rc = restrict(lev.P, lev.blk, res)
    if l + 1 == len(hier) - 1:
        ec = coarsest_solve(hier[l + 1], rc)
    else:
        ncyc = coarse_cycles[l] if l < len(coarse_cycles) else 1

        def inner_cycle(v):
            return vcycle(hier, l + 1, v, nu_pre, nu_post, omega, coarse_cycles, coarse_solver)

        if coarse_solver == "gcr":
            ec = gcr_fixed(hier[l + 1].apply, rc, inner_cycle, ncyc)
        else:
            ec = inner_cycle(rc)
            for _ in range(ncyc - 1):
                ec = ec + inner_cycle(rc - hier[l + 1].apply(ec))
    xc = prolong(lev.P, lev.blk, ec)
    Axc = lev.apply(xc)
    alpha = minimal_residual_coefficient(Axc, res)
    e = e + alpha * xc
    res = res - alpha * Axc
    de, res = smooth(lev, res, nu_post, omega)
    return e + de


# ---------------------------------------------------------------- outer solver

def fgcr(apply, b, precond=None, tol=1e-10, restart=50, max_restarts=100):
    """Flexible GCR(restart) (Sec. 5) with modified Gram-Schmidt on w = A z.

    Stops when the true residual ||b - A x|| / ||b||, recomputed from
    scratch, is <= tol.  Returns (x, info) where info holds the iteration
    count and the true relative residual.
    """
    bnorm = np.sqrt(norm2(b))
    x = np.zeros_like(b)
    r = b.copy()
    iters = 0
    history = []
    for _ in range(max_restarts):
        Z, W = [], []
        for k in range(restart):
            z = precond(r) if precond is not None else r.copy()
            w = apply(z)
            for j in range(k):
                beta = inner(W[j], w)
                w = w - beta * W[j]
                z = z - beta * Z[j]
            nw = np.sqrt(norm2(w))
            if nw == 0.0:
                raise ArithmeticError("GCR breakdown")
            w = w / nw
            z = z / nw
            a = inner(w, r)
            x = x + a * z
            r = r - a * w
            Z.append(z)
            W.append(w)
            iters += 1
            history.append(np.sqrt(norm2(r)) / bnorm)
            if history[-1] <= tol:
                break
        r = b - apply(x)
        true_rel = np.sqrt(norm2(r)) / bnorm
        if true_rel <= tol:
            return x, {"iters": iters, "true_rel_residual": true_rel, "history": history}
    raise ArithmeticError("GCR did not converge")


def mg_solve(hier, b, tol=1e-10, restart=50, nu_pre=2, nu_post=2, omega=0.8,
             coarse_cycles=(4,), coarse_solver="gcr"):
    """MG-GCR: flexible GCR(50) preconditioned by one modified V-cycle (Sec. 5)."""
    fine = hier[0]

    def precond(r):
        return vcycle(hier, 0, r, nu_pre, nu_post, omega, coarse_cycles, coarse_solver)

    return fgcr(fine.apply, b, precond, tol, restart)
