// Level-0 operator: the 4D SU(3) Wilson-Dirac stencil (dslash).
//
// Sec. 1 (Eq. 1.1 and the paragraph after it) of Clark et al., "The removal
// of critical slowing down": D = Dslash + m with central covariant
// differences and a second-order Wilson term (r = 1, spacing 1):
//   (D psi)(n) = (4 + m) psi(n)
//     - 1/2 sum_mu [(1 - g_mu) U_mu(n) psi(n+mu) + (1 + g_mu) U_mu(n-mu)^+ psi(n-mu)].
// The kernels compute   out = a * in + b * Hop(in) + c * y
// where Hop(in)(n) = sum_mu [(1 - g_mu) U psi(n+mu) + (1 + g_mu) U^+ psi(n-mu)],
// so D = (a = 4 + m, b = -1/2) and the residual y - D x = (a = -(4 + m),
// b = +1/2, c = 1).  Optionally they also reduce <out|z> and ||out||^2 per
// right-hand side (used by the MR smoother, the alpha step and GCR).
//
// GB300 design: one thread per site and right-hand side (or two right-hand
// sides sharing each link).  Fields use the chunked level-0 layout of
// wilson_hop.cuh, so a neighbour's spinor is three 16-byte loads in
// FP16/BF16 (six in FP32) and each load of a warp is one contiguous
// transaction.  In the chiral basis every (1 -+ g_mu) has rank 2 and its
// projection is a sum of +-1 / +-i multiples of two spin components, so each
// hop multiplies one 3x3 link into two colour vectors only.  FP32/FP16/BF16
// links store two rows (12 reals) and rebuild the third as conj(row0 x row1)
// (exact for SU(3)); FP64 links keep all 18 reals because FP64 arithmetic,
// not memory, bounds the FP64 stencil on this part.  The FP32-arithmetic
// stencil runs its SU(3) products as paired FP32 FMAs over the two projected
// spin rows (one instruction per two products): with 16-bit storage the
// stencil is bound by the FP32 pipes, not by HBM, on this part.
#include "common.cuh"
#include "kernels.h"
#include "wilson_hop.cuh"

namespace wmg {

template <typename S, typename G, int NL>
struct WilsonArgs {
  const S* in;
  S* out;
  const S* y;  // may be null
  const S* z;  // dot partner, may be null (then no reduction)
  const G* U;  // links, layout of wilson_hop.cuh
  int L[4];
  int V;
  double a, b, c;
  size_t vstride;  // complex elements per right-hand side (12 V)
  RedArgs red;
  const double* adiag;  // null, or per right-hand side multiplier of a
};

__device__ __forceinline__ void site_coords(int s, const int (&L)[4], int (&c)[4], int (&stride)[4]) {
  int q = s;
  c[0] = q % L[0];
  q /= L[0];
  c[1] = q % L[1];
  q /= L[1];
  c[2] = q % L[2];
  c[3] = q / L[2];
  stride[0] = 1;
  stride[1] = L[0];
  stride[2] = L[0] * L[1];
  stride[3] = stride[2] * L[2];
}

// Hopping term of NR right-hand sides at one site: FP32 arithmetic in paired
// form (Acc2), FP64 in the scalar form.
template <typename R, int NR>
struct HopAcc;
template <int NR>
struct HopAcc<float, NR> {
  Acc2 a[NR];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < NR; ++r) acc2_zero(a[r]);
  }
  template <int MU, bool FWD>
  __device__ __forceinline__ void add(int r, const cx<float> (&psi)[12], const Link<float>& u) {
    hop_packed<MU, FWD>(a[r], psi, u);
  }
  __device__ __forceinline__ cx<float> get(int r, int c) const { return acc2_get(a[r], c); }
};
template <int NR>
struct HopAcc<double, NR> {
  cx<double> a[NR][4][3];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int k = 0; k < 3; ++k) a[r][sp][k] = wmg::zero<double>();
  }
  template <int MU, bool FWD>
  __device__ __forceinline__ void add(int r, const cx<double> (&psi)[12], const Link<double>& u) {
    hop_vals<MU, FWD, double>(a[r], psi, u);
  }
  __device__ __forceinline__ cx<double> get(int r, int c) const { return a[r][c / 3][c % 3]; }
};

// The two hops of direction MU for NR right-hand sides: each link is loaded
// (and its third row rebuilt) once and applied to every right-hand side.
template <int MU, int NR, typename R, typename S, typename G, int NL>
__device__ __forceinline__ void hop_pair(HopAcc<R, NR>& acc, const WilsonArgs<S, G, NL>& A, const S* in, int s,
                                         const int (&c)[4], const int (&stride)[4]) {
  const int L = A.L[MU], st = stride[MU];
  const int fwd = (c[MU] == L - 1) ? s - (L - 1) * st : s + st;
  const int bwd = (c[MU] == 0) ? s + (L - 1) * st : s - st;
  Link<R> u;
  load_link<R, G, NL>(u, A.U, MU, A.V, s);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    cx<R> psi[12];
    ld_spinor<R, S>(in + r * A.vstride, A.V, fwd, psi);
    acc.template add<MU, true>(r, psi, u);
  }
  load_link<R, G, NL>(u, A.U, MU, A.V, bwd);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    cx<R> psi[12];
    ld_spinor<R, S>(in + r * A.vstride, A.V, bwd, psi);
    acc.template add<MU, false>(r, psi, u);
  }
}

// Own-site part of chunk j of a site's output for one right-hand side
// (pointers offset to it): out = ca in + cb h + cc y, with the dot partials of
// the value as stored against z.  y or z may alias out, so they are read
// through the L2 (coherent with this thread's earlier stores).
template <typename R, typename S>
__device__ __forceinline__ void finish_chunk(const cx<R> (&h)[4], int j, const S* in, S* out, const S* y, const S* z,
                                             size_t V, int s, R ca, R cb, R cc, R (&red)[3]) {
  const size_t i0 = (size_t)(((unsigned)j * (unsigned)V + (unsigned)s) << 2);
  cx<R> xin[4], yv[4], v[4];
  ld_chunk<R, S>(in, i0, xin);
  if (y) ld_chunk_cg<R, S>(y, i0, yv);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = mk<R>(fma(cb, h[k].re, ca * xin[k].re), fma(cb, h[k].im, ca * xin[k].im));
    if (y) v[k] = mk<R>(fma(cc, yv[k].re, v[k].re), fma(cc, yv[k].im, v[k].im));
  }
  st_chunk<S, R>(out, i0, v);
  if (z) {
    // reduce the value as stored, so dots see exactly the vector kept
    cx<R> zz[4];
    ld_chunk_cg<R, S>(z, i0, zz);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const cx<R> vs = as_stored<S>(v[k]);
      const cx<R> d = cmul_conj(vs, zz[k]);
      red[0] += d.re;
      red[1] += d.im;
      red[2] += norm2(vs);
    }
  }
}

template <typename R, typename S, typename HA>
__device__ __forceinline__ void finish_site(const HA& acc, int r, const S* in, S* out, const S* y, const S* z, size_t V,
                                            int s, R ca, R cb, R cc, R (&red)[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    cx<R> h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = acc.get(r, 4 * j + k);
    finish_chunk<R, S>(h, j, in, out, y, z, V, s, ca, cb, cc, red);
  }
}

// Thread = (site, NR consecutive right-hand sides).  Every right-hand side's
// output and dot partials are computed with the same operations in the same
// order for any NT and NR, and the dots of right-hand side r are reduced over
// the same CTAs of NT sites, so a launch shape never changes a result bit.
// DOTS: the launch reduces <out|z>, ||out||^2 (then every thread of a CTA
// takes part in the reduction); without it threads past the lattice leave at
// once and no reduction code runs.
template <typename S, typename G, int NL, int NT, int NR, bool DOTS>
__device__ __forceinline__ void wilson_body(const WilsonArgs<S, G, NL>& A) {
  typedef typename Store<S>::R R;
  const int V = A.V;
  const int s = blockIdx.x * NT + threadIdx.x;
  const int rhs0 = blockIdx.y * NR;
  const S* in = A.in + rhs0 * A.vstride;
  R red[NR][3];  // per-thread partial dots in the arithmetic type
#pragma unroll
  for (int r = 0; r < NR; ++r) red[r][0] = red[r][1] = red[r][2] = (R)0;
  if (!DOTS && s >= V) return;
  if (s < V) {
    int c[4], stride[4];
    site_coords(s, A.L, c, stride);
    HopAcc<R, NR> acc;
    acc.zero();
    hop_pair<0, NR>(acc, A, in, s, c, stride);
    hop_pair<1, NR>(acc, A, in, s, c, stride);
    hop_pair<2, NR>(acc, A, in, s, c, stride);
    hop_pair<3, NR>(acc, A, in, s, c, stride);
    const R cb = (R)A.b, cc = (R)A.c;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const R ca = (R)(A.adiag ? A.a * A.adiag[rhs0 + r] : A.a);
      const size_t ro = (size_t)(rhs0 + r) * A.vstride;
      finish_site<R, S>(acc, r, A.in + ro, A.out + ro, A.y ? A.y + ro : nullptr, DOTS ? A.z + ro : nullptr,
                        (size_t)V, s, ca, cb, cc, red[r]);
    }
  }
  if (DOTS) {
#pragma unroll
    for (int r = 0; r < NR; ++r) grid_reduce<3, NT, R>(red[r], A.red, rhs0 + r);
  }
}

// The plain single-right-hand-side form (no dots) on 16-bit fields is bound
// by the FP32 pipes: its register budget is capped so that 512 threads fit
// on an SM.  The other forms keep the compiler's own choice (with FP32
// fields more registers keep more loads in flight, which is what that
// memory-bound form needs).
template <typename S, typename G, int NL, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) wilson_plain_kernel(const WilsonArgs<S, G, NL> A) {
  wilson_body<S, G, NL, NT, 1, false>(A);
}
template <typename S, typename G, int NL, int NT, int NR, bool DOTS>
__global__ void __launch_bounds__(NT) wilson_kernel(const WilsonArgs<S, G, NL> A) {
  wilson_body<S, G, NL, NT, NR, DOTS>(A);
}

// Small lattices (a few thousand sites): one thread per site leaves most of
// the GPU idle, so a CTA of 8 warps takes 32 sites and warp w computes hop
// w (direction w / 2, forward for even w) for all 32 of them; the eight
// partial sums of each site are then added in direction order through shared
// memory and warps 0-2 finish one four-component chunk each (output, y term
// and fused dots).  Deterministic; a different association of the same terms
// than the one-thread-per-site kernel.
template <int MU, bool FWD, typename R, typename G, int NL, typename In>
__device__ __forceinline__ void one_hop(cx<R> (&acc)[4][3], const G* U, int V, const In& in, int s, const int (&c)[4],
                                        const int (&stride)[4], int L) {
  const int st = stride[MU];
  Link<R> u;
  cx<R> psi[12];
  if (FWD) {
    const int nb = (c[MU] == L - 1) ? s - (L - 1) * st : s + st;
    load_link<R, G, NL>(u, U, MU, V, s);
    in(nb, psi);
  } else {
    const int nb = (c[MU] == 0) ? s + (L - 1) * st : s - st;
    load_link<R, G, NL>(u, U, MU, V, nb);
    in(nb, psi);
  }
  hop_vals<MU, FWD, R>(acc, psi, u);
}

// Input of a hop: the 12 components of a site of a stored field.
template <typename R, typename S>
struct StoredIn {
  const S* p;
  size_t V;
  __device__ __forceinline__ void operator()(int site, cx<R> (&v)[12]) const { ld_spinor<R, S>(p, V, site, v); }
};

// The hop of warp w (direction w / 2, forward for even w) into the CTA's partial sums.
template <typename R, typename G, int NL, typename In>
__device__ __forceinline__ void warp_hop(R (&part)[8][24][32], const G* U, const int (&Lat)[4], int V, const In& in,
                                         int s, bool valid) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cx<R> acc[4][3];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[sp][a] = zero<R>();
  if (valid) {
    int c[4], stride[4];
    site_coords(s, Lat, c, stride);
    switch (warp) {  // uniform across the warp
      case 0: one_hop<0, true, R, G, NL>(acc, U, V, in, s, c, stride, Lat[0]); break;
      case 1: one_hop<0, false, R, G, NL>(acc, U, V, in, s, c, stride, Lat[0]); break;
      case 2: one_hop<1, true, R, G, NL>(acc, U, V, in, s, c, stride, Lat[1]); break;
      case 3: one_hop<1, false, R, G, NL>(acc, U, V, in, s, c, stride, Lat[1]); break;
      case 4: one_hop<2, true, R, G, NL>(acc, U, V, in, s, c, stride, Lat[2]); break;
      case 5: one_hop<2, false, R, G, NL>(acc, U, V, in, s, c, stride, Lat[2]); break;
      case 6: one_hop<3, true, R, G, NL>(acc, U, V, in, s, c, stride, Lat[3]); break;
      default: one_hop<3, false, R, G, NL>(acc, U, V, in, s, c, stride, Lat[3]); break;
    }
  }
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      part[warp][2 * (sp * 3 + a)][lane] = acc[sp][a].re;
      part[warp][2 * (sp * 3 + a) + 1][lane] = acc[sp][a].im;
    }
}

// Chunk j of the hopping term of this lane's site, summed over the eight hops in order.
template <typename R>
__device__ __forceinline__ void warp_hop_sum(const R (&part)[8][24][32], int j, cx<R> (&h)[4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int comp = 4 * j + k;
    h[k] = zero<R>();
#pragma unroll
    for (int w = 0; w < 8; ++w) h[k] = h[k] + mk<R>(part[w][2 * comp][lane], part[w][2 * comp + 1][lane]);
  }
}

template <typename S, typename G, int NL>
__global__ void __launch_bounds__(256) wilson_small_kernel(const WilsonArgs<S, G, NL> A) {
  typedef typename Store<S>::R R;
  __shared__ R part[8][24][32];  // [hop][real component][site of the CTA]
  const int V = A.V;
  const int warp = threadIdx.x >> 5;
  const int s = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rhs = blockIdx.y;
  const size_t ro = (size_t)rhs * A.vstride;
  warp_hop<R, G, NL>(part, A.U, A.L, V, StoredIn<R, S>{A.in + ro, (size_t)V}, s, s < V);
  __syncthreads();
  R red[3] = {(R)0, (R)0, (R)0};
  if (warp < 3 && s < V) {
    const R ca = (R)(A.adiag ? A.a * A.adiag[rhs] : A.a), cb = (R)A.b, cc = (R)A.c;
    cx<R> h[4];
    warp_hop_sum<R>(part, warp, h);
    finish_chunk<R, S>(h, warp, A.in + ro, A.out + ro, A.y ? A.y + ro : nullptr, A.z ? A.z + ro : nullptr,
                       (size_t)V, s, ca, cb, cc, red);
  }
  if (A.z) grid_reduce<3, 256, R>(red, A.red, rhs);
}

// Site x right-hand-side counts up to which the warp-per-hop kernel runs.
constexpr int kSmallSites = 32768;

// ------------------------------------------------------------------ MR-fused stencil
// One MR step (Sec. 3) that also finishes the previous step's update (the
// setup relaxation of Sec. 2 on small lattices).  With c = omega <p|r>/<p|p>
// of the previous step (per right-hand side, from its reduction slot) and
// that step's update direction u (null: u = r):
//   x = xin + c u,   r' = r - c p,   out = a r' + b Hop(r') (= A r'),
// with <out|r'>, ||out||^2 reduced for the next step.  r' at the neighbours
// is formed on the fly from r and p with the same operations, and rounded to
// the storage type the same way, as at their own sites, so every site sees
// the r' that is stored; each thread stores r' and x at its own site.
template <typename R, typename S>
struct ShiftedIn {
  const S* r;
  const S* p;
  size_t V;
  cx<R> c;
  __device__ __forceinline__ void operator()(int site, cx<R> (&v)[12]) const {
    cx<R> pv[12];
    ld_spinor<R, S>(r, V, site, v);
    ld_spinor<R, S>(p, V, site, pv);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = as_stored<S>(v[k] - c * pv[k]);
  }
};

struct MrFuseArgs {
  const void* pprev;
  const void* u;    // null: u = r
  const void* xin;  // null: x starts from 0
  void* x;
  void* rout;
  const double* dots;
  int dstride;
  double omega;
};

// c of right-hand side rhs, once per CTA in FP64 from the FP64 slot (as the MR update kernel forms it).
template <typename R>
__device__ __forceinline__ cx<R> fused_coef(const MrFuseArgs& F, int rhs) {
  __shared__ double sc[2];
  if (threadIdx.x == 0) {
    const double* d = F.dots + (size_t)rhs * F.dstride;
    const double den = d[2];
    double cr = 0.0, ci = 0.0;
    if (den > 0.0 && isfinite(den)) {
      cr = F.omega * d[0] / den;
      ci = F.omega * d[1] / den;
    }
    sc[0] = cr;
    sc[1] = ci;
  }
  __syncthreads();
  return mk<R>((R)sc[0], (R)sc[1]);
}

// Own-site part of chunk j of a fused step for one right-hand side (offset
// ro): x and r' stored, out = a r' + b h, and the dot partials of out
// against r'.
template <typename R, typename S>
__device__ __forceinline__ void fused_chunk(const MrFuseArgs& F, const ShiftedIn<R, S>& in, S* out, size_t ro, int j,
                                            int s, const cx<R> (&h)[4], R ca, R cb, R (&red)[3]) {
  const size_t i0 = (j * in.V + s) << 2;
  cx<R> rv[4], pv[4], uv[4], xv[4], v[4];
  ld_chunk<R, S>(in.r, i0, rv);
  ld_chunk<R, S>(in.p, i0, pv);
  if (F.u) ld_chunk<R, S>((const S*)F.u + ro, i0, uv);
  if (F.xin) ld_chunk<R, S>((const S*)F.xin + ro, i0, xv);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const cx<R> rn = as_stored<S>(rv[k] - in.c * pv[k]);
    if (!F.xin) xv[k] = zero<R>();
    xv[k] = cfma(in.c, F.u ? uv[k] : rv[k], xv[k]);
    rv[k] = rn;
    v[k] = cb * h[k];
    v[k] = v[k] + ca * rn;
  }
  st_chunk<S, R>((S*)F.x + ro, i0, xv);
  st_chunk<S, R>((S*)F.rout + ro, i0, rv);
  st_chunk<S, R>(out, i0, v);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const cx<R> vs = as_stored<S>(v[k]);
    const cx<R> d = cmul_conj(vs, rv[k]);
    red[0] += d.re;
    red[1] += d.im;
    red[2] += norm2(vs);
  }
}

// One thread per site and right-hand side (the hop order of the scalar hop).
template <typename S, typename G, int NL, int NT>
__global__ void __launch_bounds__(NT) wilson_mr_kernel(const WilsonArgs<S, G, NL> A, const MrFuseArgs F) {
  typedef typename Store<S>::R R;
  const int V = A.V;
  const int s = blockIdx.x * NT + threadIdx.x;
  const int rhs = blockIdx.y;
  const cx<R> cf = fused_coef<R>(F, rhs);
  const size_t ro = (size_t)rhs * A.vstride;
  const ShiftedIn<R, S> in{A.in + ro, (const S*)F.pprev + ro, (size_t)V, cf};
  R red[3] = {(R)0, (R)0, (R)0};
  if (s < V) {
    int c[4], stride[4];
    site_coords(s, A.L, c, stride);
    cx<R> acc[4][3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) acc[sp][a] = zero<R>();
    one_hop<0, true, R, G, NL>(acc, A.U, V, in, s, c, stride, A.L[0]);
    one_hop<0, false, R, G, NL>(acc, A.U, V, in, s, c, stride, A.L[0]);
    one_hop<1, true, R, G, NL>(acc, A.U, V, in, s, c, stride, A.L[1]);
    one_hop<1, false, R, G, NL>(acc, A.U, V, in, s, c, stride, A.L[1]);
    one_hop<2, true, R, G, NL>(acc, A.U, V, in, s, c, stride, A.L[2]);
    one_hop<2, false, R, G, NL>(acc, A.U, V, in, s, c, stride, A.L[2]);
    one_hop<3, true, R, G, NL>(acc, A.U, V, in, s, c, stride, A.L[3]);
    one_hop<3, false, R, G, NL>(acc, A.U, V, in, s, c, stride, A.L[3]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<R> h[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) h[k] = acc[(4 * j + k) / 3][(4 * j + k) % 3];
      fused_chunk<R, S>(F, in, A.out + ro, ro, j, s, h, (R)A.a, (R)A.b, red);
    }
  }
  grid_reduce<3, NT, R>(red, A.red, rhs);
}

// Small lattices: the warp-per-hop layout of wilson_small_kernel.
template <typename S, typename G, int NL>
__global__ void __launch_bounds__(256) wilson_small_mr_kernel(const WilsonArgs<S, G, NL> A, const MrFuseArgs F) {
  typedef typename Store<S>::R R;
  __shared__ R part[8][24][32];
  const int V = A.V;
  const int warp = threadIdx.x >> 5;
  const int s = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rhs = blockIdx.y;
  const cx<R> cf = fused_coef<R>(F, rhs);
  const size_t ro = (size_t)rhs * A.vstride;
  const ShiftedIn<R, S> in{A.in + ro, (const S*)F.pprev + ro, (size_t)V, cf};
  warp_hop<R, G, NL>(part, A.U, A.L, V, in, s, s < V);
  __syncthreads();
  R red[3] = {(R)0, (R)0, (R)0};
  if (warp < 3 && s < V) {
    cx<R> h[4];
    warp_hop_sum<R>(part, warp, h);
    fused_chunk<R, S>(F, in, A.out + ro, ro, warp, s, h, (R)A.a, (R)A.b, red);
  }
  grid_reduce<3, 256, R>(red, A.red, rhs);
}
template <typename S, typename G, int NL>
static int launch_mr_t(const DslashCall& d, const MrFuseArgs& F, cudaStream_t st) {
  WilsonArgs<S, G, NL> A;
  A.in = (const S*)d.in;
  A.out = (S*)d.out;
  A.y = nullptr;
  A.z = nullptr;
  A.U = (const G*)d.links;
  for (int k = 0; k < 4; ++k) A.L[k] = d.L[k];
  A.V = d.L[0] * d.L[1] * d.L[2] * d.L[3];
  A.a = d.a;
  A.b = d.b;
  A.c = 0.0;
  A.vstride = (size_t)12 * A.V;
  A.red = d.red;
  A.adiag = nullptr;
  if constexpr (NL != 9) {
    if ((size_t)A.V * d.nrhs <= (size_t)kSmallSites) {  // the same split as the unfused stencil
      wilson_small_mr_kernel<S, G, NL><<<dim3((A.V + 31) / 32, d.nrhs), 256, 0, st>>>(A, F);
      return launch_ok() ? 0 : -1;
    }
  }
  wilson_mr_kernel<S, G, NL, 128><<<dim3((A.V + 127) / 128, d.nrhs), 128, 0, st>>>(A, F);
  return launch_ok() ? 0 : -1;
}

template <typename S, typename G, int NL, int NT, int NR>
static int launch_nt(const WilsonArgs<S, G, NL>& A, int nrhs, cudaStream_t st) {
  dim3 grid((A.V + NT - 1) / NT, nrhs / NR);
  if (A.z) {
    wilson_kernel<S, G, NL, NT, NR, true><<<grid, NT, 0, st>>>(A);
  } else {
    if constexpr (NR == 1 && sizeof(S) == 4)
      wilson_plain_kernel<S, G, NL, NT><<<grid, NT, 0, st>>>(A);
    else
      wilson_kernel<S, G, NL, NT, NR, false><<<grid, NT, 0, st>>>(A);
  }
  return launch_ok() ? 0 : -1;
}

// Launch shapes (threads per CTA NT, right-hand sides per thread NR), in the
// order a tuner sees them: with fused dots NT stays 128 (the reduction's
// association depends on the CTA size), NR = 2 needs an even count; FP64 has
// the one default shape (its stencil is bound by FP64 arithmetic).
struct WShape {
  int nt, nr;
};
static const WShape kShapesDots[] = {{128, 1}, {128, 2}};
static const WShape kShapesFree[] = {{128, 1}, {64, 1}, {256, 1}, {128, 2}, {64, 2}, {256, 2}};

int wilson_variants(int prec, bool dots, int nrhs, int V) {
  if (prec == 0 || (size_t)V * nrhs <= (size_t)kSmallSites) return 1;  // one shape: FP64, or the small-lattice kernel
  const bool even = nrhs % 2 == 0;
  if (dots) return even ? 2 : 1;
  return even ? 6 : 3;
}

template <typename S, typename G, int NL>
static int launch_t(const DslashCall& d, cudaStream_t st) {
  WilsonArgs<S, G, NL> A;
  A.in = (const S*)d.in;
  A.out = (S*)d.out;
  A.y = (const S*)d.y;
  A.z = (const S*)d.z;
  A.U = (const G*)d.links;
  for (int k = 0; k < 4; ++k) A.L[k] = d.L[k];
  A.V = d.L[0] * d.L[1] * d.L[2] * d.L[3];
  A.a = d.a;
  A.b = d.b;
  A.c = d.c;
  A.vstride = (size_t)12 * A.V;
  A.red = d.red;
  A.adiag = d.adiag;
  if constexpr (NL == 9) {
    return launch_nt<S, G, NL, 128, 1>(A, d.nrhs, st);
  } else {
    if ((size_t)A.V * d.nrhs <= (size_t)kSmallSites) {  // small lattice: a warp per hop
      dim3 grid((A.V + 31) / 32, d.nrhs);
      wilson_small_kernel<S, G, NL><<<grid, 256, 0, st>>>(A);
      return launch_ok() ? 0 : -1;
    }
    WShape sh = {128, 1};
    if (d.variant >= 0 && d.variant < wilson_variants(1, d.z != nullptr, d.nrhs, A.V))
      sh = d.z ? kShapesDots[d.variant] : kShapesFree[d.variant];
    if (sh.nr == 2) {
      if (sh.nt == 64) return launch_nt<S, G, NL, 64, 2>(A, d.nrhs, st);
      if (sh.nt == 256) return launch_nt<S, G, NL, 256, 2>(A, d.nrhs, st);
      return launch_nt<S, G, NL, 128, 2>(A, d.nrhs, st);
    }
    if (sh.nt == 64) return launch_nt<S, G, NL, 64, 1>(A, d.nrhs, st);
    if (sh.nt == 256) return launch_nt<S, G, NL, 256, 1>(A, d.nrhs, st);
    return launch_nt<S, G, NL, 128, 1>(A, d.nrhs, st);
  }
}

int launch_wilson_mr(const DslashCall& d, const void* pprev, const void* u, const void* xin, void* x, void* rout,
                     const double* dots, int dstride, double omega, cudaStream_t st) {
  const MrFuseArgs F{pprev, u, xin, x, rout, dots, dstride, omega};
  switch (d.prec) {
    case 0: return launch_mr_t<double2, double2, 9>(d, F, st);
    case 1: return launch_mr_t<float2, float2, 6>(d, F, st);
    case 2: return launch_mr_t<__half2, __half2, 6>(d, F, st);
    case 3: return launch_mr_t<__nv_bfloat162, __nv_bfloat162, 6>(d, F, st);
  }
  return -1;
}

// CTAs per right-hand side of a launch with fused dots (sizes the reduction partials).
int wilson_blocks(int V) { return V <= kSmallSites ? (V + 31) / 32 : (V + 127) / 128; }

int launch_wilson(const DslashCall& d, cudaStream_t st) {
  switch (d.prec) {
    case 0: return launch_t<double2, double2, 9>(d, st);
    case 1: return launch_t<float2, float2, 6>(d, st);
    case 2: return launch_t<__half2, __half2, 6>(d, st);
    case 3: return launch_t<__nv_bfloat162, __nv_bfloat162, 6>(d, st);
  }
  return -1;
}


// ------------------------------------------------------------------ links
// External gauge layout [4][V][3][3] complex FP64 -> the internal link layout
// of wilson_hop.cuh in the storage precision (NL = 9 for FP64, 6 = two rows
// otherwise).
template <typename G, int NL>
__global__ void pack_links_kernel(const double2* __restrict__ ext, G* __restrict__ out, int V) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over 4 V sites x NL
  const size_t tot = (size_t)4 * V * NL;
  if (i >= tot) return;
  const int site = (int)(i % V);
  const int k = (int)((i / V) % NL);
  const int mu = (int)(i / ((size_t)V * NL));
  double2 v = ext[((size_t)mu * V + site) * 9 + k];
  stc(out, lidx<G, NL>(mu, k, site, V), mk<double>(v.x, v.y));
}

// ------------------------------------------------------------------ link check
// Largest deviation of an external FP64 gauge field [4][V][3][3] from SU(3):
// max over links of |U U^+ - 1| and |det U - 1| (largest real or imaginary
// part).  A non-negative float's bits order like the float, so the maximum
// goes through an integer atomicMax; NaN counts as infinite.
__global__ void su3_check_kernel(const double2* __restrict__ ext, size_t nlinks, unsigned* worst) {
  unsigned best = 0u;
  for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += (size_t)gridDim.x * blockDim.x) {
    cx<double> u[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double2 v = ext[l * 9 + i * 3 + j];
        u[i][j] = mk<double>(v.x, v.y);
      }
    double dev = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        cx<double> g = zero<double>();
#pragma unroll
        for (int k = 0; k < 3; ++k) g = cfma_conj(u[j][k], u[i][k], g);  // (U U^+)_ij
        if (i == j) g.re -= 1.0;
        dev = fmax(dev, fmax(fabs(g.re), fabs(g.im)));
      }
    const cx<double> det = u[0][0] * (u[1][1] * u[2][2] - u[1][2] * u[2][1]) -
                           u[0][1] * (u[1][0] * u[2][2] - u[1][2] * u[2][0]) +
                           u[0][2] * (u[1][0] * u[2][1] - u[1][1] * u[2][0]);
    dev = fmax(dev, fmax(fabs(det.re - 1.0), fabs(det.im)));
    const unsigned bits = (dev == dev) ? __float_as_uint((float)dev) : 0x7f800000u;
    best = bits > best ? bits : best;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned other = __shfl_down_sync(0xffffffffu, best, o);
    best = other > best ? other : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(worst, best);
}

int launch_su3_check(const void* ext, int V, unsigned* worst, cudaStream_t st) {
  const size_t n = (size_t)4 * V;
  size_t nb = (n + 255) / 256;
  if (nb > 1216) nb = 1216;
  su3_check_kernel<<<(unsigned)(nb < 1 ? 1 : nb), 256, 0, st>>>((const double2*)ext, n, worst);
  return launch_ok() ? 0 : -1;
}

int launch_pack_links(int prec, const void* ext, void* out, int V, cudaStream_t st) {
  const int NL = prec == 0 ? 9 : 6;
  const size_t tot = (size_t)4 * V * NL;
  const int nt = 256;
  const unsigned nb = (unsigned)((tot + nt - 1) / nt);
  switch (prec) {
    case 0: pack_links_kernel<double2, 9><<<nb, nt, 0, st>>>((const double2*)ext, (double2*)out, V); break;
    case 1: pack_links_kernel<float2, 6><<<nb, nt, 0, st>>>((const double2*)ext, (float2*)out, V); break;
    case 2: pack_links_kernel<__half2, 6><<<nb, nt, 0, st>>>((const double2*)ext, (__half2*)out, V); break;
    case 3:
      pack_links_kernel<__nv_bfloat162, 6><<<nb, nt, 0, st>>>((const double2*)ext, (__nv_bfloat162*)out, V);
      break;
    default: return -1;
  }
  return launch_ok() ? 0 : -1;
}

}  // namespace wmg
