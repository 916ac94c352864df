/*
 * wilson_mg.h -- C ABI of the GB300 adaptive-multigrid solver for the 4D SU(3)
 * Wilson-Dirac system D x = b.
 *
 * Paper: M. A. Clark, J. Brannick, R. C. Brower, S. F. McCormick,
 * T. A. Manteuffel, J. C. Osborn, C. Rebbi, "The removal of critical slowing
 * down", Lattice 2008 (arXiv:0811.4331).
 *
 * Operator (Sec. 1, Eq. 1.1 and the paragraph after it), lattice spacing 1,
 * Wilson parameter r = 1, periodic boundaries:
 *   (D psi)(n) = (4 + m) psi(n)
 *       - 1/2 sum_mu [(1 - gamma_mu) U_mu(n) psi(n+mu) + (1 + gamma_mu) U_mu(n-mu)^+ psi(n-mu)]
 * with the chiral gamma basis gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]
 * (k = x, y, z), gamma_t = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1).
 *
 * ---------------------------------------------------------------- layouts
 * Complex numbers are interleaved (re, im).  dims = {Lx, Ly, Lz, Lt}; the
 * site index is lexicographic with x fastest:
 *   site = x + Lx * (y + Ly * (z + Lz * t)),  V = Lx Ly Lz Lt.
 * EXTERNAL layouts (what mg_setup / mg_solve / the field converters take):
 *   gauge   : double complex [4][V][3][3]  (mu = x, y, z, t; row, column)
 *   spinor  : double complex [nrhs][V][4][3]  (spin, colour) = [nrhs][V][12]
 *   level-l field (l >= 1): double complex [nrhs][V_l][2 Nv_l]; components
 *             [0, Nv_l) have chirality +, [Nv_l, 2 Nv_l) chirality -.
 * INTERNAL layout (what dslash_apply / coarse_apply / restrict / prolong /
 * mr_apply operate on, in the precision named by `prec`):
 *   level 0: [nrhs][3][V][4] complex, element (r, c, s) at
 *            r * 12 V + ((c / 4) V + s) 4 + c % 4 (c = spin * 3 + colour):
 *            three chunks of four components, each chunk site-major, so one
 *            site's chunk is a single 16-byte load in FP16 / BF16;
 *   level l >= 1: component-major [nrhs][ncomp][V_l] complex, element
 *            (r, c, s) at (r * ncomp + c) * V_l + s, ncomp = 2 Nv_l.
 * Complex element types: MG_F64 = 2 x double, MG_F32 = 2 x float,
 * MG_F16 = 2 x IEEE binary16, MG_BF16 = 2 x bfloat16.  mg_field_to_internal /
 * mg_field_from_internal convert between the two.
 *
 * ---------------------------------------------------------------- conventions
 * Every call returns an mg_status.  No exception crosses the ABI.  On error
 * mg_last_error() returns a static, thread-local message.  `stream` is a
 * cudaStream_t (NULL = legacy default stream); all device work of a call is
 * enqueued on it.  Calls that take or return host data, or that return
 * results to the host (mg_setup, mg_solve, the getters), synchronise the
 * stream before returning; the *_apply calls do not.  A handle is not
 * thread-safe.  Device pointers passed in must stay valid until the work
 * enqueued on `stream` has finished.
 */
#ifndef WILSON_MG_H
#define WILSON_MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_EINVAL = 1,      /* bad argument: sizes, level, precision, layout, null pointer */
  MG_ENOMEM = 2,      /* device allocation failed */
  MG_ECUDA = 3,       /* a CUDA call failed (message in mg_last_error) */
  MG_ERANK = 4,       /* block Gram-Schmidt lost rank (a candidate fell below 1e-12 of its norm) */
  MG_ENOCONV = 5,     /* solver hit max_iter; x holds the last iterate, stats its true residual */
  MG_EBREAKDOWN = 6,  /* GCR breakdown (||A z|| = 0) */
  MG_ENAN = 7         /* a residual norm became NaN or Inf */
} mg_status;

typedef enum { MG_F64 = 0, MG_F32 = 1, MG_F16 = 2, MG_BF16 = 3 } mg_precision;

#define MG_MAX_LEVELS 4

/* Solver parameters.  mg_default_params fills the paper's choices:
 * V(2,2) (Sec. 4, Sec. 5), omega = 0.8 (Sec. 3), 4 next-level V-cycles per
 * fine coarse correction (Sec. 5), GCR(50) (Sec. 5), 4^4 blocks (Sec. 3,
 * Sec. 5), Nv = 20 (Sec. 5). */
typedef struct {
  int n_levels;                       /* 1 = no preconditioner (plain GCR), 2..MG_MAX_LEVELS */
  int block[MG_MAX_LEVELS - 1][4];    /* aggregate of level l -> l+1, {bx, by, bz, bt} */
  int nv[MG_MAX_LEVELS - 1];          /* null vectors of level l (coarse ncomp = 2 nv) */
  int setup_sweeps[MG_MAX_LEVELS - 1];/* MR steps on A x = 0 per candidate (Sec. 2, "l") */
  int coarse_cycles[MG_MAX_LEVELS - 1];/* next-level V-cycles per coarse correction of level l (at most 8
                                         with the flexible coarse solver) */
  int nu_pre, nu_post;                /* MR smoothing steps before / after the coarse correction */
  double omega;                       /* MR under-relaxation */
  int gcr_restart;                    /* outer flexible GCR restart length */
  int max_iter;                       /* outer GCR iteration cap (all restarts) */
  int mixed;                          /* 0 = plain FP64 everywhere; 1 = mixed precision */
  int fine_prec;                      /* mixed: storage of level-0 smoother work (MG_F16/MG_BF16/MG_F32) */
  int coarse_prec;                    /* mixed: storage of levels 1..L-1 (MG_F32, or fine_prec itself) */
  double reliable_delta;              /* mixed: inner FP32 GCR reduces ||r|| by this factor before an FP64 update */
  uint64_t seed;                      /* on-device start vectors: level l uses stream seed + l */
  int use_graphs;                     /* 1: replay the V-cycle as a captured CUDA graph; 0: launch eagerly */
  int coarse_mma;                     /* mixed: 1 = coarse stencils of levels 1..L-2 on tensor cores (BF16
                                         operator in MMA fragment order, FP32 accumulation) */
  int coarse_solver;                  /* the coarse_cycles applications of the next level's V-cycle:
                                         0 = as steps of flexible GCR preconditioned by it (default),
                                         1 = as stationary sweeps e += V(r - A e) */
  int adapt_steps;                    /* adaptive steps of Sec. 2 per level: the first nv - adapt_nv[l]
                                         candidates come from relaxation; each step appends a batch of the
                                         rest, made by the current solver (flexible GCR preconditioned by the
                                         level's multigrid cycle, restarted every 8 iterations) applied to
                                         A x = 0 from random starts, and rebuilds P and the levels below
                                         (default 0: relaxation only) */
  int adapt_cycles;                   /* solver iterations per adaptive candidate (default 16) */
  int adapt_nv[MG_MAX_LEVELS - 1];    /* candidates of level l made by the adaptive steps, < nv[l] */
  int defer_coarsest;                 /* 1: mg_setup leaves the coarsest inverse to the first solve on this
                                         handle (for a hierarchy that only feeds mg_retarget_batch, which
                                         builds every retargeted inverse in shared launches); ignored with
                                         adaptive steps, which need it during setup (default 0) */
  int fine_smoother;                  /* level-0 smoother of the cycle: 0 = MR on D (Sec. 3, default);
                                         1 = even-odd (not in the paper): the nu_pre / nu_post MR steps
                                         run on the Schur complement S of the even sites (see
                                         schur_apply) from zero, then the odd sites are solved exactly;
                                         needs every lattice extent even */
  int coarsest_f64;                   /* mixed: 1 = the coarsest inverse in FP64 and the coarsest solve in FP64
                                         (no refinement); 0 = an FP32 inverse with one FP64 refinement step
                                         (default).  Plain hierarchies are FP64 throughout */
} mg_params;

/* Per right-hand side solve statistics. */
typedef struct {
  int iters;                 /* outer GCR iterations */
  int restarts;              /* GCR restarts */
  int reliable_updates;      /* FP64 true-residual recomputations (mixed) */
  long long fine_dslash;     /* level-0 operator applications, all precisions */
  long long fine_dslash_f64; /* of which in FP64 */
  double true_rel_residual;  /* ||b - D x|| / ||b||, recomputed in FP64 at exit */
  double solve_seconds;      /* wall time of this right-hand side's solve */
} mg_stats;

typedef struct mg_handle mg_handle;

/* Last error message of this thread (never NULL). */
const char* mg_last_error(void);

/* Fill `p` with defaults: 2 levels, 4^4 blocks, Nv = 20, 20 setup sweeps,
 * V(2,2), omega 0.8, 4 coarse cycles, GCR(50), max_iter 2000, plain FP64,
 * CUDA graphs on. */
int mg_default_params(mg_params* p);

/* Build the solver for gauge field `gauge` and mass `mass`.
 *   h            : out, a new handle owning every device buffer of the hierarchy.
 *   gauge        : external layout, FP64; host memory if gauge_on_device == 0,
 *                  device memory otherwise.  Copied; the caller keeps ownership.
 *   dims         : {Lx, Ly, Lz, Lt}, each >= 1, at most 2^26 sites in all.
 *   p            : parameters (copied).  For every level l < n_levels - 1 the
 *                  level's extent must be divisible by block[l],
 *                  nv[l] <= (components per chirality) * (sites per block),
 *                  and one block of a P column (components x sites, complex
 *                  in the setup's precision: FP64 plain, FP32 mixed) must fit
 *                  the Galerkin product's 200 KB of shared memory (a 4^4
 *                  fine block in FP64 takes 48 KB).
 *   starts       : NULL, or an array of n_levels - 1 host pointers; starts[l]
 *                  holds nv[l] FP64 start vectors of level l in the external
 *                  layout [nv][V_l][ncomp_l].  NULL entries (or NULL starts)
 *                  use the on-device counter generator (seed p->seed + l).
 * Setup per level (Sec. 2 adaptive steps 1-3, Eq. 2.3; Sec. 3): setup_sweeps
 * MR steps (omega) on A x = 0 from each start, unit-normalise, blockwise
 * FP64 modified Gram-Schmidt (two passes, candidate order) per aggregate and
 * chirality into P, then A_{l+1} = P^+ A_l P as a 9-point stencil of
 * 2Nv x 2Nv blocks; the coarsest level gets a dense inverse (FP64 plain;
 * FP32 mixed, applied with one FP64 refinement step).
 * Errors: MG_EINVAL (also when a link deviates from SU(3), max |U U^+ - 1|
 * or |det U - 1| above 1e-10: the FP32 / 16-bit operators store two rows and
 * rebuild the third as for SU(3)), MG_ENOMEM, MG_ERANK, MG_ECUDA.  On error
 * *h is NULL. */
int mg_setup(mg_handle** h, const double* gauge, int gauge_on_device, const int dims[4],
             double mass, const mg_params* p, const double* const* starts, void* stream);

/* A new handle for mass `mass` that reuses the null vectors of `src`.
 * D(m) = D(0) + m 1 has the same eigenvectors at every mass (Sec. 1), so the
 * near-null space found by the setup of `src` serves any mass; and since
 * P^+ P = 1 on every level (Eq. 2.3), A_l(m) = A_l(m_src) + (m - m_src) 1 for
 * every Galerkin operator A_l = P^+ A_{l-1} P (Sec. 2).  The new handle owns
 * device copies of the links, prolongators and coarse stencils of `src`
 * (shifted), and its own coarsest inverse, rebuilt for `mass`.  `src` is
 * not modified and stays valid.  Errors as mg_setup. */
int mg_retarget(const mg_handle* src, double mass, mg_handle** h, void* stream);

/* mg_retarget for `count` (1..64) masses at once: h[z] gets masses[z].  The
 * coarsest inverses of all of them are built by one batched elimination
 * (every pivot step of every matrix in one launch).  On error no handle is
 * returned (h[z] = NULL). */
int mg_retarget_batch(const mg_handle* src, const double* masses, int count, mg_handle** h, void* stream);

/* Release every device buffer of `h` (NULL is allowed) into the library's
 * memory cache (mg_trim_cache).  Synchronises the device first: no work on
 * any stream may still use the handle. */
int mg_destroy(mg_handle* h);

/* Solve D x_r = b_r for r = 0..nrhs-1 to ||b - D x|| / ||b|| <= tol with
 * flexible GCR(gcr_restart) preconditioned by one modified multigrid V-cycle
 * (Sec. 5), or unpreconditioned when n_levels == 1.
 *   b, x  : external spinor layout, FP64, [nrhs][V][12]; device memory if
 *           on_device != 0, else host memory.  x is the initial guess on
 *           entry (zero it for none) and the solution on return.
 *   stats : NULL or an array of nrhs mg_stats.
 * Every returned x is checked against its true FP64 residual, recomputed at exit.
 * Errors: MG_EINVAL, MG_ENOCONV (x and stats still filled), MG_EBREAKDOWN,
 * MG_ENAN, MG_ECUDA. */
int mg_solve(mg_handle* h, const double* b, double* x, int nrhs, int on_device, double tol,
             mg_stats* stats, void* stream);

/* One multi-right-hand-side solve in which right-hand side r has its own mass
 * masses[r] (a mass sweep as one solve).  D(m) = D(0) + m 1 (Sec. 1) and
 * P^+ P = 1 (Eq. 2.3) make every level's operator at m_r the handle's plus
 * (m_r - mass) on the diagonal, applied per right-hand side inside the
 * stencil kernels; the coarsest solve takes the inverse of its own mass
 * (built for the distinct masses on first use and kept until other masses
 * come).  The handle's null vectors serve every mass (as for mg_retarget).
 * b, x, nrhs (1..64), on_device, tol, stats as mg_solve.  Not with the
 * even-odd smoother.  Errors: MG_EINVAL, and those of mg_solve. */
int mg_solve_masses(mg_handle* h, const double* masses, const double* b, double* x, int nrhs, int on_device,
                    double tol, mg_stats* stats, void* stream);

/* mg_solve on `count` distinct handles at once (e.g. one hierarchy per mass
 * of a sweep, Sec. 5): handle i solves b[i] -> x[i] (nrhs right-hand sides
 * each, layouts and on_device as mg_solve) on its own host thread and stream
 * (streams[i], or a stream created for the call when streams is NULL), so
 * the kernels of independent latency-bound solves run side by side on the
 * GPU.  Not in the paper; each solve's arithmetic, and so its result, is
 * that of mg_solve alone.  stats: NULL or count * nrhs entries, handle-major.
 * Returns when every solve has finished; on failure, the first failing
 * handle's status, with "handle i: " before its message.
 * Errors: MG_EINVAL (also for a repeated handle), and those of mg_solve. */
int mg_solve_many(mg_handle* const* hs, int count, const double* const* b, double* const* x, int nrhs,
                  int on_device, double tol, mg_stats* stats, void* const* streams);

/* Unpreconditioned Krylov solvers on level 0 alone: the methods the paper
 * measures multigrid against (Secs. 4-5).
 *   method : MG_KRYLOV_BICGSTAB -- BiCGstab (van der Vorst 1992) on D x = b;
 *            MG_KRYLOV_CGNR     -- CG on D^+ D x = D^+ b, D^+ = gamma5 D gamma5;
 *            MG_KRYLOV_*_EO     -- the same method on the even-odd Schur system
 *              S x_e = b_e + H_eo b_o / (2M) (see schur_apply; not in the
 *              paper), then x_o = (b_o + H_oe x_e / 2) / M.  The full residual
 *              of the reconstructed x equals the Schur residual, so the Schur
 *              solve stops at tol ||b||; needs every lattice extent even.
 *              stats.fine_dslash counts one per S application (two half-
 *              lattice hops = one full stencil's work).
 *   FP64 throughout on the handle's FP64 links (any handle: the hierarchy is
 *   not used); one right-hand side after the other; b, x, nrhs, on_device,
 *   tol, stats as mg_solve (stats.iters = iterations, stats.fine_dslash =
 *   operator applications); a recursive residual below tol is confirmed by
 *   the true residual, else the method restarts from it.
 * Errors: MG_EINVAL, MG_ENOCONV after max_iter iterations (x and stats
 * filled), MG_ENAN, MG_ECUDA. */
#define MG_KRYLOV_BICGSTAB 0
#define MG_KRYLOV_CGNR 1
#define MG_KRYLOV_BICGSTAB_EO 2
#define MG_KRYLOV_CGNR_EO 3
int krylov_solve(mg_handle* h, int method, const double* b, double* x, int nrhs, int on_device, double tol,
                 int max_iter, mg_stats* stats, void* stream);

/* out = D in on level 0 (Sec. 1 operator above) for nrhs internal-layout
 * spinors of precision `prec` (device memory; in and out must not overlap).
 * Arithmetic is FP64 for MG_F64 and FP32 otherwise.  Errors: MG_EINVAL. */
int dslash_apply(mg_handle* h, int prec, const void* in, void* out, int nrhs, void* stream);

/* ---------------------------------------------------------------- even-odd
 * Not in the paper: the standard Schur-complement (red-black) reduction of
 * the Sec. 1 operator.  With M = 4 + m and H the hopping term (D = M - H/2),
 * H links only sites of opposite parity p(n) = (x + y + z + t) mod 2, so
 *   D = [[M, -H_eo/2], [-H_oe/2, M]],   S = M - H_eo H_oe / (4 M)
 * is the Schur complement on the even sites, gamma5-Hermitian like D.
 * HALF layout: the level-0 internal layout on the V/2 sites of one parity,
 * [nrhs][3][V/2][4] complex in precision prec, the sites in lexicographic
 * order (half index = site / 2).  Every lattice extent must be even
 * (MG_EINVAL otherwise).  Device memory; the calls do not synchronise; the
 * parity-major link copy of precision prec is made on the first call (one
 * more link array of 4 NL V complex, held by the handle). */

/* Split nrhs internal-layout level-0 spinors into their even and odd halves. */
int eo_split(mg_handle* h, int prec, const void* full, void* even, void* odd, int nrhs, void* stream);
/* full = merge(even, odd); a NULL half is taken as zero. */
int eo_merge(mg_handle* h, int prec, const void* even, const void* odd, void* full, int nrhs, void* stream);
/* out = a x + b H_{p,1-p} in on half fields: out and x (NULL: no a-term) have
 * parity `parity_out`, in the other parity.  Arithmetic as dslash_apply.
 * in and out must not overlap; x may equal out only if in does not. */
int dslash_eo_apply(mg_handle* h, int prec, int parity_out, const void* x, const void* in, void* out, double a,
                    double b, int nrhs, void* stream);
/* out = S in on even half fields (two half-lattice hops; an odd half
 * scratch is taken from the handle's work vectors). */
int schur_apply(mg_handle* h, int prec, const void* in, void* out, int nrhs, void* stream);

/* out = A_level in for the coarse stencil operator of `level` >= 1
 * (A_l = P^+ A_{l-1} P, Sec. 2), internal layout, device memory.
 * Precisions: the vector storage; the operator is held in the same
 * precision, except that with coarse_mma an FP32 call runs on tensor cores
 * with the operator in BF16 (FP32 accumulation).
 * Errors: MG_EINVAL (no such level / precision). */
int coarse_apply(mg_handle* h, int level, int prec, const void* in, void* out, int nrhs,
                 void* stream);

/* out (level l+1) = P_l^+ in (level l)  -- restriction R = P^+ (Sec. 3).
 * Internal layouts, precision `prec` for both vectors (MG_F64 or MG_F32). */
int restrict_apply(mg_handle* h, int level, int prec, const void* in, void* out, int nrhs,
                   void* stream);

/* out (level l) = P_l in (level l+1)  -- prolongation (Sec. 2). */
int prolong_apply(mg_handle* h, int level, int prec, const void* in, void* out, int nrhs,
                  void* stream);

/* `steps` under-relaxed MR steps (Sec. 3, omega from the params) on
 * A_level x = b starting from x (internal layout, precision prec; x is
 * updated in place, r receives b - A x as updated by the iteration). */
int mr_apply(mg_handle* h, int level, int prec, const void* b, void* x, void* r, int steps,
             void* stream);

/* e = M r: one modified V-cycle of the hierarchy applied to the level-0
 * internal-layout FP64 residual r (plain FP64 hierarchy only). */
int vcycle_apply(mg_handle* h, const void* r, void* e, void* stream);

/* Copy nrhs FP64 external-layout fields of `level` (host if on_device == 0)
 * to the internal layout in precision prec on the device, and back. */
int mg_field_to_internal(mg_handle* h, int level, int prec, const double* ext, int on_device,
                         void* internal, int nrhs, void* stream);
int mg_field_from_internal(mg_handle* h, int level, int prec, const void* internal,
                           double* ext, int on_device, int nrhs, void* stream);

/* Sizes of level `level`: sites, components per site, null vectors (0 on
 * the coarsest level). */
int mg_level_info(mg_handle* h, int level, int dims_out[4], int* ncomp, int* nv);

/* Copy the FP64 prolongator of level l to host memory, external layout
 * [nv][V_l][ncomp_l]: vector k holds, on every aggregate B and chirality
 * chi, column chi * nv + k of P restricted to B (Eq. 2.3). */
int mg_get_prolongator(mg_handle* h, int level, double* out);

/* Copy the FP64 coarse stencil of level l >= 1 to host memory as
 * [9][V_l][ncomp][ncomp] complex (row i, column j); direction d = 0 is the
 * site itself, d = 1 + 2 mu the hop to n + mu, d = 2 + 2 mu to n - mu. */
int mg_get_coarse_op(mg_handle* h, int level, double* out);

/* Copy the dense inverse of the coarsest operator (Sec. 4: the coarsest
 * level is solved exactly) to host memory as [N][N] complex, N = V_c ncomp_c,
 * rows and columns in the external order (site-major, component fastest);
 * FP64 or FP32 values as the handle stores them, widened to double.  Builds
 * a deferred inverse first.  MG_EINVAL for a one-level handle. */
int mg_get_coarsest_inverse(mg_handle* h, double* out);

/* Same as mr_apply (for nrhs = 1), but allocates nothing, for callers that
 * cannot allocate device memory when they call it: a server that fixed its
 * device footprint at start-up, or a thread that must not enter the driver's
 * allocation path while other streams run.  mr_apply takes its scratch (the
 * work vector A r and the reduction partial sums, ticket counter and result
 * slot) from buffers the handle allocates on demand; this entry point takes
 * it from one fixed array of 16 MiB compiled into the library, which every
 * GPU that loads the library holds until the process exits.  The paper has
 * no counterpart.
 *   - The level's scratch (one vector of the level in `prec`, plus the
 *     reduction partials: 3 doubles per thread block of the operator kernel,
 *     or 4 per block of the separate dot pass where a coarse level in FP32
 *     runs on the tensor-core stencil, plus 512 bytes) must fit in 16 MiB,
 *     else MG_EINVAL and a message naming the sizes (an FP64 level-0 vector
 *     alone is 192 bytes per site).
 *   - It runs the operator kernels mr_apply runs for the same handle, level
 *     and precision (the tensor-core stencil on such a coarse level), in
 *     their default launch shapes; every shape gives the same bits.
 *   - The first call on a device looks up the array's device address once
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; the call zeroes the ticket counter it needs before using it.
 *     Calls whose work overlaps on the GPU (other streams, other threads)
 *     race on the array: serialise them.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine.
 * Arguments, layouts and the result are those of mr_apply. */
int mr_apply_noalloc(mg_handle* h, int level, int prec, const void* b, void* x, void* r, int steps,
                     void* stream);

/* Kernel classes of the profiler. */
typedef enum {
  MG_K_DSLASH = 0,   /* level-0 Wilson stencil */
  MG_K_COARSE = 1,   /* coarse 9-point stencil */
  MG_K_RESTRICT = 2, /* P^+ */
  MG_K_PROLONG = 3,  /* P */
  MG_K_VECTOR = 4,   /* MR / GCR vector updates, dots, conversions */
  MG_K_COARSEST = 5, /* dense coarsest solve */
  MG_K_SETUP = 6,    /* start vectors, block Gram-Schmidt, prolongator columns, copies */
  MG_K_GALERKIN = 7, /* Galerkin build of the coarse stencil */
  MG_K_INVERSE = 8,  /* dense coarsest inverse (the whole elimination as one interval) */
  MG_K_GRAM = 9,     /* Gram-Schmidt of the outer GCR (multi-dot + update, both passes as one interval) */
  MG_K_CLASSES = 10
} mg_kernel_class;

/* Enable (mask != 0, bit c = class c) or disable the per-launch profiler
 * of handle h and clear its counters.  While enabled, every launch of a
 * selected class is bracketed by two CUDA events recorded on the stream it
 * runs on (no extra synchronisation), and the V-cycle is launched eagerly
 * rather than replayed as a graph.  h == NULL sets the mask that handles
 * created afterwards start with (so that mg_setup itself is profiled). */
int mg_profile(mg_handle* h, unsigned mask);

/* Synchronise and return the number of launches and their summed event
 * time (milliseconds) of class `kclass` with storage precision `prec`
 * since the last mg_profile call. */
int mg_profile_read(mg_handle* h, int kclass, int prec, long long* launches, double* ms);

/* The algorithmic bytes of the same launches: every operand of a profiled
 * scope counted once (a stencil's matrix or links once per launch, each
 * right-hand side's vectors once), so bytes / time is the bandwidth that the
 * scope achieved against its compulsory traffic.  Classes without a count
 * (setup, Galerkin, inverse) report 0. */
int mg_profile_bytes(mg_handle* h, int kclass, int prec, double* bytes);

/* Launch-shape tuner (no counterpart in the paper).  Kernels with several
 * launch shapes -- the dslash without fused dots (threads per CTA), the
 * tensor-core coarse stencil and the tensor-core restriction / prolongation
 * (right-hand sides per CTA) -- are timed once per (kernel, precision, sizes,
 * right-hand sides) on first use outside graph capture, writing scratch
 * outputs only, and the fastest shape is kept for the process.  All shapes
 * of a kernel give bit-identical results, so the tuner changes speed only.
 * mode: 0 = off (default shapes), 1 = on (the default), 2 = forget every
 * choice and turn on, 3 / 4 = force the last / first shape of every kernel
 * (for testing that all shapes agree).  Returns the previous mode, or -1 for
 * a bad mode. */
int mg_tune(int mode);

/* Text report of the tuner's choices, one line per key:
 * "<kernel>|<precision>|<sizes...>|<rhs> <chosen shape> <us of shape 0> ...".
 * Writes at most cap - 1 characters and a NUL into buf (if buf != NULL and
 * cap > 0); returns the length of the whole report. */
int mg_tune_report(char* buf, int cap);

/* Number of kernels this library has launched since it was loaded, over
 * all handles and threads (a monotonic counter). */
unsigned long long mg_launch_count(void);

/* Number of device buffers this library has taken since it was loaded, from
 * the driver or from its cache of freed buffers, over all handles and threads
 * (a monotonic counter; frees do not lower it).  Lets a caller check that a
 * call allocated nothing. */
unsigned long long mg_alloc_count(void);

/* Device memory that handles free (mg_destroy, temporaries) is kept in a
 * process-wide cache by size class and reused by later handles, so building
 * hierarchies repeatedly does not call the driver's allocator each time.
 * mg_trim_cache synchronises the device, hands every cached block back to
 * the driver and returns the bytes freed.  Call it between solves only. */
size_t mg_trim_cache(void);

/* Device bytes the handle holds now (hierarchy, work vectors, solver
 * buffers; capacities of its buffers), for admission by memory budget. */
size_t mg_handle_bytes(const mg_handle* h);

/* Hand the handle's solve buffers (Krylov basis, work vectors of every
 * level, the inverses of mg_solve_masses) back to the memory cache, keeping
 * the hierarchy (links, prolongators, coarse operators, coarsest inverse);
 * the next solve takes them again.  Synchronises `stream` (the stream of the
 * handle's last solve; NULL: the legacy stream) first.  Returns the bytes
 * released.  A server calls it after each batch so that a resident handle
 * holds only its hierarchy between batches. */
size_t mg_release_work(mg_handle* h, void* stream);

/* Device bytes that mg_setup + mg_solve(nrhs) need for these sizes, with
 * nrhs distinct masses for mg_solve_masses (one coarsest inverse each). */
size_t mg_footprint(const int dims[4], const mg_params* p, int nrhs);

#ifdef __cplusplus
}
#endif
#endif
