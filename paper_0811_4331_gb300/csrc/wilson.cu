// Level-0 operator: the 4D SU(3) Wilson-Dirac stencil (dslash).
//
// Sec. 1 (Eq. 1.1 and the paragraph after it) of Clark et al., "The removal
// of critical slowing down": D = Dslash + m with central covariant
// differences and a second-order Wilson term (r = 1, spacing 1):
//   (D psi)(n) = (4 + m) psi(n)
//     - 1/2 sum_mu [(1 - g_mu) U_mu(n) psi(n+mu) + (1 + g_mu) U_mu(n-mu)^+ psi(n-mu)].
// The kernel computes   out = a * in + b * Hop(in) + c * y
// where Hop(in)(n) = sum_mu [(1 - g_mu) U psi(n+mu) + (1 + g_mu) U^+ psi(n-mu)],
// so D = (a = 4 + m, b = -1/2) and the residual y - D x = (a = -(4 + m),
// b = +1/2, c = 1).  Optionally it also reduces <out|z> and ||out||^2 per
// right-hand side (used by the MR smoother, the alpha step and GCR).
//
// GB300 design: one thread per site and right-hand side; spinors and links
// are component-major ([comp][site]) so each of the 12 spinor loads and 6/9
// link loads of a warp is one coalesced 128-512 byte transaction.  In the
// chiral basis every (1 -+ g_mu) has rank 2 and its projection is a sum of
// +-1 / +-i multiples of two spin components, so each hop multiplies one 3x3
// link into two colour vectors only.  FP32/FP16/BF16 links store two rows
// (12 reals) and rebuild the third as conj(row0 x row1) (exact for SU(3));
// FP64 links keep all 18 reals because FP64 arithmetic, not memory, bounds
// the FP64 stencil on this part.
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
  const G* U;  // [4][NL][V]
  int L[4];
  int V;
  double a, b, c;
  size_t vstride;  // complex elements per right-hand side (12 V)
  RedArgs red;
};

template <int MU, typename R, typename S, typename G, int NL>
__device__ __forceinline__ void hop_pair(cx<R> (&acc)[4][3], const WilsonArgs<S, G, NL>& A, const S* in,
                                         int s, const int (&c)[4], const int (&stride)[4]) {
  const int L = A.L[MU], st = stride[MU];
  const int fwd = (c[MU] == L - 1) ? s - (L - 1) * st : s + st;
  const int bwd = (c[MU] == 0) ? s + (L - 1) * st : s - st;
  Link<R> u;
  load_link<R, G, NL>(u, A.U, MU, A.V, s);
  hop<MU, true>(acc, in, A.V, fwd, u);
  load_link<R, G, NL>(u, A.U, MU, A.V, bwd);
  hop<MU, false>(acc, in, A.V, bwd, u);
}

template <typename S, typename G, int NL, int NT>
__global__ void __launch_bounds__(NT) wilson_kernel(const WilsonArgs<S, G, NL> A) {
  typedef typename Store<S>::R R;
  const int V = A.V;
  const int s = blockIdx.x * NT + threadIdx.x;
  const int rhs = blockIdx.y;
  const S* in = A.in + rhs * A.vstride;
  R acc3[3] = {(R)0, (R)0, (R)0};  // per-thread partial dots in the arithmetic type
  if (s < V) {
    int c[4], stride[4];
    {
      int q = s;
      c[0] = q % A.L[0];
      q /= A.L[0];
      c[1] = q % A.L[1];
      q /= A.L[1];
      c[2] = q % A.L[2];
      c[3] = q / A.L[2];
      stride[0] = 1;
      stride[1] = A.L[0];
      stride[2] = A.L[0] * A.L[1];
      stride[3] = stride[2] * A.L[2];
    }
    cx<R> acc[4][3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) acc[sp][a] = zero<R>();
    hop_pair<0>(acc, A, in, s, c, stride);
    hop_pair<1>(acc, A, in, s, c, stride);
    hop_pair<2>(acc, A, in, s, c, stride);
    hop_pair<3>(acc, A, in, s, c, stride);
    const R ca = (R)A.a, cb = (R)A.b, cc = (R)A.c;
    S* out = A.out + rhs * A.vstride;
    const S* y = A.y ? A.y + rhs * A.vstride : nullptr;
    const S* z = A.z ? A.z + rhs * A.vstride : nullptr;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const size_t i = (size_t)(sp * 3 + a) * V + s;
        cx<R> v = cb * acc[sp][a];
        v = v + ca * ldc<R>(in, i);
        if (y) v = v + cc * ldc<R>(y, i);
        stc(out, i, v);
        if (z) {
          // reduce the value as stored, so dots see exactly the vector kept
          cx<R> vs = as_stored<S>(v);
          cx<R> zz = ldc<R>(z, i);
          cx<R> d = cmul_conj(vs, zz);
          acc3[0] += d.re;
          acc3[1] += d.im;
          acc3[2] += norm2(vs);
        }
      }
  }
  if (A.z) grid_reduce<3, NT, R>(acc3, A.red, rhs);
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
  constexpr int NT = 128;
  dim3 grid((A.V + NT - 1) / NT, d.nrhs);
  wilson_kernel<S, G, NL, NT><<<grid, NT, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int wilson_blocks(int V) { return (V + 127) / 128; }

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
// External gauge layout [4][V][3][3] complex FP64 -> internal [4][NL][V] in
// the storage precision (NL = 9 for FP64, 6 = two rows otherwise).
template <typename G, int NL>
__global__ void pack_links_kernel(const double2* __restrict__ ext, G* __restrict__ out, int V) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over 4 V sites x NL
  const size_t tot = (size_t)4 * V * NL;
  if (i >= tot) return;
  const int site = (int)(i % V);
  const int k = (int)((i / V) % NL);
  const int mu = (int)(i / ((size_t)V * NL));
  double2 v = ext[((size_t)mu * V + site) * 9 + k];
  stc(out, i, mk<double>(v.x, v.y));
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
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace wmg
