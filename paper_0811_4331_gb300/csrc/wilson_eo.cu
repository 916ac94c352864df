// Even-odd (red-black) form of the level-0 Wilson stencil.
//
// The hopping term of the Sec. 1 operator, D = (4 + m) - 1/2 H, only links
// sites of opposite parity p(n) = (x + y + z + t) mod 2.  Splitting a field
// into its even and odd sites turns D into [[M, -H_eo/2], [-H_oe/2, M]]
// (M = 4 + m), and eliminating the odd sites leaves the Schur complement
// S = M - H_eo H_oe / (4 M) on the even sites; the odd sites then follow
// from one more hop.  This file holds the half-lattice pieces:
//
//   wilson_eo_kernel : out_p = a x_p + b H_{p,1-p} in_{1-p} + c y_p, with
//                      optional <out|z>, ||out||^2 per right-hand side;
//   eo_split_kernel  : full field -> (even, odd) half fields (also used to
//                      reorder the links parity-major);
//   eo_merge_kernel  : (even, odd) -> full field, optionally added to it.
//
// Half-field layout: the chunked level-0 layout of wilson_hop.cuh on V/2
// sites, [nrhs][3][V/2][4] complex, the sites of one parity in lexicographic
// order (needs an even Lx: each x-row then holds Lx/2 sites of either
// parity, and the k-th site of a parity has lexicographic index 2k or
// 2k + 1, so its half index is lex / 2).  Links: the link layout of
// wilson_hop.cuh with the site index parity-major (even sites 0..V/2-1, then
// odd), so the links a thread reads for its forward hops are contiguous
// across a warp.
#include "common.cuh"
#include "kernels.h"
#include "wilson_hop.cuh"

namespace wmg {

static inline bool launched() { return launch_ok(); }

template <typename S, typename G, int NL>
struct EoArgs {
  const S* x;   // parity of out, may be null
  const S* in;  // the other parity
  const S* y;   // parity of out, may be null
  const S* z;   // dot partner (parity of out), may be null
  S* out;
  const G* U;  // parity-major links
  int L[4];
  int V, Vh;
  int parity;  // of out
  double a, b, c;
  RedArgs red;
};

// Lexicographic site and coordinates of half index h of parity p.
__device__ __forceinline__ int eo_site(int h, int p, const int (&L)[4], int (&c)[4]) {
  const int lex0 = 2 * h;
  c[0] = lex0 % L[0];
  int q = lex0 / L[0];
  c[1] = q % L[1];
  q /= L[1];
  c[2] = q % L[2];
  c[3] = q / L[2];
  c[0] += (p + c[1] + c[2] + c[3]) & 1;
  return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]));
}

template <int MU, typename R, typename S, typename G, int NL>
__device__ __forceinline__ void eo_hop_pair(cx<R> (&acc)[4][3], const EoArgs<S, G, NL>& A, const S* in, int s, int h,
                                            const int (&c)[4], const int (&stride)[4]) {
  const int L = A.L[MU], st = stride[MU];
  const int fwd = (c[MU] == L - 1) ? s - (L - 1) * st : s + st;
  const int bwd = (c[MU] == 0) ? s + (L - 1) * st : s - st;
  Link<R> u;
  load_link<R, G, NL>(u, A.U, MU, A.V, A.parity * A.Vh + h);  // U_mu(n)
  hop<MU, true>(acc, in, A.Vh, fwd >> 1, u);
  load_link<R, G, NL>(u, A.U, MU, A.V, (1 - A.parity) * A.Vh + (bwd >> 1));  // U_mu(n - mu)
  hop<MU, false>(acc, in, A.Vh, bwd >> 1, u);
}

template <typename S, typename G, int NL, int NT>
__global__ void __launch_bounds__(NT) wilson_eo_kernel(const EoArgs<S, G, NL> A) {
  typedef typename Store<S>::R R;
  const int h = blockIdx.x * NT + threadIdx.x;
  const int rhs = blockIdx.y;
  const size_t ro = (size_t)rhs * 12 * A.Vh;
  R red[3] = {(R)0, (R)0, (R)0};
  if (h < A.Vh) {
    int c[4];
    const int s = eo_site(h, A.parity, A.L, c);
    const int stride[4] = {1, A.L[0], A.L[0] * A.L[1], A.L[0] * A.L[1] * A.L[2]};
    cx<R> acc[4][3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[sp][k] = zero<R>();
    const S* in = A.in + ro;
    eo_hop_pair<0>(acc, A, in, s, h, c, stride);
    eo_hop_pair<1>(acc, A, in, s, h, c, stride);
    eo_hop_pair<2>(acc, A, in, s, h, c, stride);
    eo_hop_pair<3>(acc, A, in, s, h, c, stride);
    const R ca = (R)A.a, cb = (R)A.b, cc = (R)A.c;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // x, y or z may alias out: read them through the L2 (coherent with this thread's stores)
      const size_t i0 = ro + (((size_t)j * A.Vh + h) << 2);
      cx<R> xv[4], yv[4], v[4];
      if (A.x) ld_chunk_cg<R, S>(A.x, i0, xv);
      if (A.y) ld_chunk_cg<R, S>(A.y, i0, yv);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = 4 * j + k;
        v[k] = cb * acc[c / 3][c % 3];
        if (A.x) v[k] = v[k] + ca * xv[k];
        if (A.y) v[k] = v[k] + cc * yv[k];
      }
      st_chunk<S, R>(A.out, i0, v);
      if (A.z) {
        cx<R> zz[4];
        ld_chunk_cg<R, S>(A.z, i0, zz);
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
  }
  if (A.z) grid_reduce<3, NT, R>(red, A.red, rhs);
}

constexpr int kEoThreads = 128;

int eo_blocks(int V) { return (V / 2 + kEoThreads - 1) / kEoThreads; }

template <typename S, typename G, int NL>
static int launch_eo_t(const EoCall& d, cudaStream_t st) {
  EoArgs<S, G, NL> A;
  A.x = (const S*)d.x;
  A.in = (const S*)d.in;
  A.y = (const S*)d.y;
  A.z = (const S*)d.z;
  A.out = (S*)d.out;
  A.U = (const G*)d.links;
  for (int k = 0; k < 4; ++k) A.L[k] = d.L[k];
  A.V = d.L[0] * d.L[1] * d.L[2] * d.L[3];
  A.Vh = A.V / 2;
  A.parity = d.parity;
  A.a = d.a;
  A.b = d.b;
  A.c = d.c;
  A.red = d.red;
  dim3 grid(eo_blocks(A.V), d.nrhs);
  wilson_eo_kernel<S, G, NL, kEoThreads><<<grid, kEoThreads, 0, st>>>(A);
  return launched() ? 0 : -1;
}

int launch_wilson_eo(const EoCall& d, cudaStream_t st) {
  if (d.L[0] % 2 || d.L[1] % 2 || d.L[2] % 2 || d.L[3] % 2 || (d.parity & ~1)) return -1;
  switch (d.prec) {
    case 0: return launch_eo_t<double2, double2, 9>(d, st);
    case 1: return launch_eo_t<float2, float2, 6>(d, st);
    case 2: return launch_eo_t<__half2, __half2, 6>(d, st);
    case 3: return launch_eo_t<__nv_bfloat162, __nv_bfloat162, 6>(d, st);
  }
  return -1;
}

// ------------------------------------------------------------------ split / merge
// Thread (h, row): lexicographic sites 2h and 2h + 1 of the row are one even
// and one odd site (the parity of 2h is that of y + z + t).  Rows are
// right-hand side x component (or mu x link element); the halves of row r
// start at even + r * hstride and odd + r * hstride.
template <typename T>
__global__ void eo_split_kernel(const T* __restrict__ full, T* __restrict__ even, T* __restrict__ odd, int L0, int L1,
                                int L2, int Vh, size_t hstride) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= Vh) return;
  const size_t row = blockIdx.y;
  const int lex0 = 2 * h;
  int q = lex0 / L0;
  const int y = q % L1;
  q /= L1;
  const int z = q % L2, t = q / L2;
  const int odd_first = (y + z + t) & 1;
  const T* f = full + row * (size_t)(2 * Vh) + lex0;
  const T a = f[0], b = f[1];
  even[row * hstride + h] = odd_first ? b : a;
  odd[row * hstride + h] = odd_first ? a : b;
}

// full = (add ? full : 0) + merge(even, odd) on chunked level-0 fields (rows
// of V four-component chunks); a null half is zero.
template <typename S>
__global__ void eo_merge_kernel(const S* __restrict__ even, const S* __restrict__ odd, S* full, int L0, int L1, int L2,
                                int Vh, int add) {
  typedef typename Store<S>::R R;
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= Vh) return;
  const size_t row = blockIdx.y;
  const int lex0 = 2 * h;
  int q = lex0 / L0;
  const int y = q % L1;
  q /= L1;
  const int z = q % L2, t = q / L2;
  const int odd_first = (y + z + t) & 1;
  // rows of 4-complex chunks (one chunk of one site per element)
  const size_t hi = (row * (size_t)Vh + h) << 2;
  const size_t fe = (row * (size_t)(2 * Vh) + lex0 + odd_first) << 2;
  const size_t fo = (row * (size_t)(2 * Vh) + lex0 + 1 - odd_first) << 2;
  cx<R> ve[4], vo[4];
  if (even) ld_chunk<R, S>(even, hi, ve);
  if (odd) ld_chunk<R, S>(odd, hi, vo);
  cx<R> fv[4], gv[4];
  if (add) {
    ld_chunk_cg<R, S>(full, fe, fv);
    ld_chunk_cg<R, S>(full, fo, gv);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!even) ve[k] = zero<R>();
    if (!odd) vo[k] = zero<R>();
    if (add) {
      ve[k] = ve[k] + fv[k];
      vo[k] = vo[k] + gv[k];
    }
  }
  st_chunk<S, R>(full, fe, ve);
  st_chunk<S, R>(full, fo, vo);
}

template <typename T>
static int split_t(const void* full, void* even, void* odd, const int L[4], size_t rows, size_t hstride,
                   cudaStream_t st) {
  const int Vh = L[0] * L[1] * L[2] * L[3] / 2;
  dim3 grid((Vh + 255) / 256, (unsigned)rows);
  eo_split_kernel<T><<<grid, 256, 0, st>>>((const T*)full, (T*)even, (T*)odd, L[0], L[1], L[2], Vh, hstride);
  return launched() ? 0 : -1;
}

struct alignas(16) Bytes32 {
  uint4 a, b;
};
struct alignas(16) Bytes64 {
  uint4 a, b, c, d;
};

int launch_eo_split(size_t elem_bytes, const void* full, void* even, void* odd, const int L[4], size_t rows,
                    size_t hstride, cudaStream_t st) {
  if (L[0] % 2 || rows == 0 || rows > 65535) return -1;
  switch (elem_bytes) {
    case 64: return split_t<Bytes64>(full, even, odd, L, rows, hstride, st);
    case 32: return split_t<Bytes32>(full, even, odd, L, rows, hstride, st);
    case 16: return split_t<uint4>(full, even, odd, L, rows, hstride, st);
    case 8: return split_t<float2>(full, even, odd, L, rows, hstride, st);
    case 4: return split_t<unsigned>(full, even, odd, L, rows, hstride, st);
  }
  return -1;
}

// Links in the layout of wilson_hop.cuh -> the same with the sites parity-major:
// every run of V site-indexed elements is split into its even and odd halves.
int launch_eo_links(int prec, const void* links, void* out, const int L[4], cudaStream_t st) {
  const size_t V = (size_t)L[0] * L[1] * L[2] * L[3], Vh = V / 2;
  const char* src = (const char*)links;
  char* dst = (char*)out;
  if (prec == 2 || prec == 3) {  // [4][V] 16-byte elements (k 0..3), then [4][V] 8-byte elements (k 4, 5)
    if (launch_eo_split(16, src, dst, dst + Vh * 16, L, 4, V, st)) return -1;
    return launch_eo_split(8, src + 64 * V, dst + 64 * V, dst + 64 * V + Vh * 8, L, 4, V, st);
  }
  if (prec == 1) return launch_eo_split(16, src, dst, dst + Vh * 16, L, 12, V, st);  // [12][V] x 16 bytes
  if (prec == 0) return launch_eo_split(16, src, dst, dst + Vh * 16, L, 36, V, st);  // [36][V] x 16 bytes
  return -1;
}

template <typename S>
static int merge_t(const void* even, const void* odd, void* full, const int L[4], size_t rows, int add,
                   cudaStream_t st) {
  const int Vh = L[0] * L[1] * L[2] * L[3] / 2;
  dim3 grid((Vh + 255) / 256, (unsigned)rows);
  eo_merge_kernel<S><<<grid, 256, 0, st>>>((const S*)even, (const S*)odd, (S*)full, L[0], L[1], L[2], Vh, add);
  return launched() ? 0 : -1;
}

int launch_eo_merge(int prec, const void* even, const void* odd, void* full, const int L[4], size_t rows, int add,
                    cudaStream_t st) {
  if (L[0] % 2 || rows == 0 || rows > 65535) return -1;
  switch (prec) {
    case 0: return merge_t<double2>(even, odd, full, L, rows, add, st);
    case 1: return merge_t<float2>(even, odd, full, L, rows, add, st);
    case 2: return merge_t<__half2>(even, odd, full, L, rows, add, st);
    case 3: return merge_t<__nv_bfloat162>(even, odd, full, L, rows, add, st);
  }
  return -1;
}

}  // namespace wmg
