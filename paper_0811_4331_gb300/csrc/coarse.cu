// Coarse-grid kernels: the coarse 9-point stencil A_c = P^+ A P (Sec. 2),
// restriction R = P^+ and prolongation P (Sec. 3, Eq. 3.2 and the text
// after it: [gamma5, P] = 0 makes R = P^+), single right-hand side and
// batched over right-hand sides on CUDA cores.
//
// Layouts.  A level-l vector is [rhs][ncomp][V] complex; the stencil is
// C[d][i][j][B] (d = 0 self, 1 + 2 mu = B + mu, 2 + 2 mu = B - mu; row i,
// column j; coarse site B fastest) so that a warp of consecutive sites reads
// one contiguous run of each matrix element.  The prolongator is stored per
// aggregate and chirality as [B][chi][k][c][s] (k < nv, c < ncomp / 2, s a
// site of the aggregate in x-fastest order): the restriction of one coarse
// component is a contiguous dot product and the prolongation of one fine
// component a contiguous column read.
#include "common.cuh"
#include "kernels.h"

namespace wmg {

static inline bool launched() { return cudaGetLastError() == cudaSuccess; }

// ------------------------------------------------------------------ apply
template <typename S>
struct CoarseArgs {
  const S* C;
  const S* in;
  S* out;
  const S* y;
  const S* z;
  int L[4];
  int V;
  int n;  // ncomp
  double a, c;
  RedArgs red;
};

template <typename S, int NT>
__global__ void __launch_bounds__(NT) coarse_apply_kernel(const CoarseArgs<S> A) {
  typedef typename Store<S>::R R;
  const int V = A.V, n = A.n;
  const int t = blockIdx.x * NT + threadIdx.x;  // t = i V + B
  const int rhs = blockIdx.y;
  const size_t voff = (size_t)rhs * n * V;
  double red[3] = {0.0, 0.0, 0.0};
  if (t < n * V) {
    const int i = t / V, B = t - i * V;
    int c[4];
    site_coords(B, A.L, c);
    cx<R> acc = zero<R>();
    for (int d = 0; d < 9; ++d) {
      const int nb = neighbor(c, A.L, d);
      const S* row = A.C + ((size_t)(d * n + i) * n) * V + B;
      const S* x = A.in + voff + nb;
      for (int j = 0; j < n; ++j) acc = cfma(ldc<R>(row, (size_t)j * V), ldc<R>(x, (size_t)j * V), acc);
    }
    const size_t o = voff + (size_t)i * V + B;
    cx<R> v = (R)A.a * acc;
    if (A.y) v = v + (R)A.c * ldc<R>(A.y, o);
    stc(A.out, o, v);
    if (A.z) {
      const cx<R> vs = as_stored<S>(v);
      const cx<R> dd = cmul_conj(vs, ldc<R>(A.z, o));
      red[0] = (double)dd.re;
      red[1] = (double)dd.im;
      red[2] = (double)norm2(vs);
    }
  }
  if (A.z) grid_reduce<3, NT>(red, A.red, rhs);
}

int launch_coarse_apply(const CoarseCall& k, cudaStream_t st) {
  constexpr int NT = 128;
  const int V = k.L[0] * k.L[1] * k.L[2] * k.L[3];
  dim3 grid((k.ncomp * V + NT - 1) / NT, k.nrhs);
#define WMG_COARSE(S)                                        \
  {                                                          \
    CoarseArgs<S> A;                                         \
    A.C = (const S*)k.C;                                     \
    A.in = (const S*)k.in;                                   \
    A.out = (S*)k.out;                                       \
    A.y = (const S*)k.y;                                     \
    A.z = (const S*)k.z;                                     \
    for (int q = 0; q < 4; ++q) A.L[q] = k.L[q];             \
    A.V = V;                                                 \
    A.n = k.ncomp;                                           \
    A.a = k.a;                                               \
    A.c = k.c;                                               \
    A.red = k.red;                                           \
    coarse_apply_kernel<S, NT><<<grid, NT, 0, st>>>(A);      \
  }
  switch (k.prec) {
    case 0: WMG_COARSE(double2); break;
    case 1: WMG_COARSE(float2); break;
    case 2: WMG_COARSE(__half2); break;
    case 3: WMG_COARSE(__nv_bfloat162); break;
    default: return -1;
  }
#undef WMG_COARSE
  return launched() ? 0 : -1;
}

int coarse_blocks(int ncomp, int V) { return (ncomp * V + 127) / 128; }

// ------------------------------------------------------------------ aggregates
// Fine site of aggregate B, aggregate-local site s.
__device__ __forceinline__ int agg_site(const Agg& g, int B, int s) {
  int cb[4], cl[4], cf[4];
  site_coords(B, g.Lc, cb);
  site_coords(s, g.blk, cl);
#pragma unroll
  for (int m = 0; m < 4; ++m) cf[m] = cb[m] * g.blk[m] + cl[m];
  return site_index(cf, g.L);
}

// r_c[(chi nv + k)][B] = sum_{c, s} conj(P[B][chi][k][c][s]) r[(chi nhalf + c)][site(B, s)]
template <typename SI, typename SP, typename SO, int NT>
__global__ void __launch_bounds__(NT) restrict_kernel(const Agg g, const SP* P, const SI* in, SO* out) {
  typedef typename Store<SP>::R R;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* sm = (cx<R>*)smem_raw;  // [ncomp][bsites]
  const int B = blockIdx.x, rhs = blockIdx.y;
  const int bs = g.bsites, nh = g.nhalf;
  const SI* vin = in + (size_t)rhs * g.ncomp * g.V;
  for (int e = threadIdx.x; e < g.ncomp * bs; e += NT) {
    const int c = e / bs, s = e - c * bs;
    sm[e] = ldc<R>(vin, (size_t)c * g.V + agg_site(g, B, s));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int len = nh * bs;
  for (int row = warp; row < 2 * g.nv; row += NT / 32) {
    const int chi = row / g.nv;
    const SP* pr = P + ((size_t)B * 2 * g.nv + row) * len;
    const cx<R>* v = sm + (size_t)chi * len;
    cx<R> acc = zero<R>();
    for (int e = lane; e < len; e += 32) acc = cfma_conj(ldc<R>(pr, e), v[e], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.re += __shfl_down_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_down_sync(0xffffffffu, acc.im, o);
    }
    if (lane == 0) stc(out, ((size_t)rhs * 2 * g.nv + row) * g.Vc + B, acc);
  }
}

// x[(chi nhalf + c)][site(B, s)] = sum_k P[B][chi][k][c][s] x_c[(chi nv + k)][B]
template <typename SI, typename SP, typename SO, int NT>
__global__ void __launch_bounds__(NT) prolong_kernel(const Agg g, const SP* P, const SI* in, SO* out) {
  typedef typename Store<SP>::R R;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* xc = (cx<R>*)smem_raw;  // [2 nv]
  const int B = blockIdx.x, rhs = blockIdx.y;
  const int bs = g.bsites, nh = g.nhalf, nv = g.nv;
  for (int q = threadIdx.x; q < 2 * nv; q += NT) xc[q] = ldc<R>(in, ((size_t)rhs * 2 * nv + q) * g.Vc + B);
  __syncthreads();
  const size_t len = (size_t)nh * bs;
  for (int e = threadIdx.x; e < g.ncomp * bs; e += NT) {
    const int c = e / bs, s = e - c * bs;
    const int chi = c / nh, cl = c - chi * nh;
    const SP* pc = P + ((size_t)B * 2 + chi) * nv * len + (size_t)cl * bs + s;
    cx<R> acc = zero<R>();
    for (int k = 0; k < nv; ++k) acc = cfma(ldc<R>(pc, (size_t)k * len), xc[chi * nv + k], acc);
    stc(out, ((size_t)rhs * g.ncomp + c) * g.V + agg_site(g, B, s), acc);
  }
}

template <typename SI, typename SP, typename SO>
static int restrict_t(const Agg& g, const void* P, const void* in, void* out, int nrhs, cudaStream_t st) {
  typedef typename Store<SP>::R R;
  constexpr int NT = 256;
  const size_t sm = (size_t)g.ncomp * g.bsites * sizeof(cx<R>);
  if (sm > 200 * 1024) return -1;
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(restrict_kernel<SI, SP, SO, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  restrict_kernel<SI, SP, SO, NT><<<dim3(g.Vc, nrhs), NT, sm, st>>>(g, (const SP*)P, (const SI*)in, (SO*)out);
  return launched() ? 0 : -1;
}

template <typename SI, typename SP, typename SO>
static int prolong_t(const Agg& g, const void* P, const void* in, void* out, int nrhs, cudaStream_t st) {
  typedef typename Store<SP>::R R;
  constexpr int NT = 256;
  const size_t sm = (size_t)2 * g.nv * sizeof(cx<R>);
  prolong_kernel<SI, SP, SO, NT><<<dim3(g.Vc, nrhs), NT, sm, st>>>(g, (const SP*)P, (const SI*)in, (SO*)out);
  return launched() ? 0 : -1;
}

// Supported (vector-in, P, vector-out) precision triples.
int launch_restrict(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                    cudaStream_t st) {
  if (pin == 0 && pP == 0 && pout == 0) return restrict_t<double2, double2, double2>(g, P, in, out, nrhs, st);
  if (pin == 1 && pP == 1 && pout == 1) return restrict_t<float2, float2, float2>(g, P, in, out, nrhs, st);
  if (pin == 2 && pP == 2 && pout == 1) return restrict_t<__half2, __half2, float2>(g, P, in, out, nrhs, st);
  if (pin == 3 && pP == 3 && pout == 1)
    return restrict_t<__nv_bfloat162, __nv_bfloat162, float2>(g, P, in, out, nrhs, st);
  if (pin == 2 && pP == 2 && pout == 2) return restrict_t<__half2, __half2, __half2>(g, P, in, out, nrhs, st);
  return -1;
}

int launch_prolong(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                   cudaStream_t st) {
  if (pin == 0 && pP == 0 && pout == 0) return prolong_t<double2, double2, double2>(g, P, in, out, nrhs, st);
  if (pin == 1 && pP == 1 && pout == 1) return prolong_t<float2, float2, float2>(g, P, in, out, nrhs, st);
  if (pin == 1 && pP == 2 && pout == 2) return prolong_t<float2, __half2, __half2>(g, P, in, out, nrhs, st);
  if (pin == 1 && pP == 3 && pout == 3)
    return prolong_t<float2, __nv_bfloat162, __nv_bfloat162>(g, P, in, out, nrhs, st);
  if (pin == 2 && pP == 2 && pout == 2) return prolong_t<__half2, __half2, __half2>(g, P, in, out, nrhs, st);
  return -1;
}

// ------------------------------------------------------------------ coarsest: dense inverse
// Dense FP64 matrix of a stencil operator in the internal vector order
// (row i V + B, column j V + B'), written into the left half of an
// augmented [N][2N] array whose right half is set to the identity.
__global__ void stencil_to_dense_kernel(const double2* C, int L0, int L1, int L2, int L3, int n, double2* aug) {
  const int L[4] = {L0, L1, L2, L3};
  const int V = L0 * L1 * L2 * L3;
  const int N = n * V;
  const size_t tot = (size_t)N * 2 * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / (2 * (size_t)N)), col = (int)(e % (2 * (size_t)N));
    double2 v = make_double2(0.0, 0.0);
    if (col < N) {
      const int i = row / V, B = row % V, j = col / V, Bp = col % V;
      int c[4];
      site_coords(B, L, c);
      for (int d = 0; d < 9; ++d) {
        if (neighbor(c, L, d) != Bp) continue;
        const double2 a = C[((size_t)(d * n + i) * n + j) * V + B];
        v.x += a.x;
        v.y += a.y;
      }
    } else if (col - N == row) {
      v.x = 1.0;
    }
    aug[e] = v;
  }
}

// Gauss-Jordan step k, part 1 (one block): partial pivot on column k, swap
// rows, scale the pivot row, save column k (zero at k) for the update.
__global__ void gj_pivot_kernel(double2* aug, int N, int k, double2* colbuf, int* err) {
  __shared__ double best[1024];
  __shared__ int arg[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t ld = 2 * (size_t)N;
  double b = -1.0;
  int a = N;
  for (int i = k + tid; i < N; i += nt) {
    const double2 v = aug[(size_t)i * ld + k];
    const double m = v.x * v.x + v.y * v.y;
    if (m > b) {
      b = m;
      a = i;
    }
  }
  best[tid] = b;
  arg[tid] = a;
  __syncthreads();
  for (int o = nt / 2; o > 0; o >>= 1) {
    if (tid < o) {
      const double b2 = best[tid + o];
      const int a2 = arg[tid + o];
      if (b2 > best[tid] || (b2 == best[tid] && a2 < arg[tid])) {
        best[tid] = b2;
        arg[tid] = a2;
      }
    }
    __syncthreads();
  }
  const int p = arg[0];
  if (!(best[0] > 0.0)) {
    if (tid == 0) *err = 1;
    return;
  }
  if (p != k) {
    for (size_t j = tid; j < ld; j += nt) {
      const double2 t = aug[(size_t)k * ld + j];
      aug[(size_t)k * ld + j] = aug[(size_t)p * ld + j];
      aug[(size_t)p * ld + j] = t;
    }
  }
  __syncthreads();
  const double2 pv = aug[(size_t)k * ld + k];
  const double den = pv.x * pv.x + pv.y * pv.y;
  const double2 inv = make_double2(pv.x / den, -pv.y / den);
  __syncthreads();
  for (size_t j = tid; j < ld; j += nt) {
    const double2 t = aug[(size_t)k * ld + j];
    aug[(size_t)k * ld + j] = make_double2(t.x * inv.x - t.y * inv.y, t.x * inv.y + t.y * inv.x);
  }
  for (int i = tid; i < N; i += nt) colbuf[i] = (i == k) ? make_double2(0.0, 0.0) : aug[(size_t)i * ld + k];
}

// Part 2: every row i != k subtracts colbuf[i] times the pivot row.
__global__ void gj_update_kernel(double2* aug, int N, int k, const double2* colbuf, const int* err) {
  if (*err) return;
  const size_t ld = 2 * (size_t)N;
  const size_t tot = (size_t)N * ld;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld);
    const size_t j = e % ld;
    if (i == k || j < (size_t)k) continue;  // columns < k of row k are already zero
    const double2 f = colbuf[i];
    const double2 pk = aug[(size_t)k * ld + j];
    double2 v = aug[e];
    v.x -= f.x * pk.x - f.y * pk.y;
    v.y -= f.x * pk.y + f.y * pk.x;
    aug[e] = v;
  }
}

__global__ void copy_right_half_kernel(const double2* aug, int N, double2* inv) {
  const size_t tot = (size_t)N * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / N, j = e % N;
    inv[e] = aug[i * 2 * (size_t)N + N + j];
  }
}

static unsigned grid_for(size_t tot, size_t cap) {
  size_t b = (tot + 255) / 256;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

int dense_inverse(const double2* C, const int L[4], int n, double2* aug, double2* colbuf, int* err, double2* inv,
                  cudaStream_t st) {
  const int V = L[0] * L[1] * L[2] * L[3];
  const int N = n * V;
  stencil_to_dense_kernel<<<grid_for((size_t)N * 2 * N, 8192), 256, 0, st>>>(C, L[0], L[1], L[2], L[3], n, aug);
  if (!launched()) return -1;
  for (int k = 0; k < N; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, st>>>(aug, N, k, colbuf, err);
    gj_update_kernel<<<grid_for((size_t)N * 2 * N, 4096), 256, 0, st>>>(aug, N, k, colbuf, err);
  }
  copy_right_half_kernel<<<grid_for((size_t)N * N, 8192), 256, 0, st>>>(aug, N, inv);
  return launched() ? 0 : -1;
}

// y = inv x for nrhs vectors; one warp per row, FP64 matrix and arithmetic.
template <typename SI, typename SO>
__global__ void dense_matvec_kernel(int N, const double2* inv, const SI* x, SO* y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int rhs = blockIdx.y;
  if (warp >= N) return;
  const double2* row = inv + (size_t)warp * N;
  const SI* xr = x + (size_t)rhs * N;
  cx<double> acc = zero<double>();
  for (int j = lane; j < N; j += 32) {
    const double2 a = row[j];
    acc = cfma(mk<double>(a.x, a.y), ldc<double>(xr, j), acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.re += __shfl_down_sync(0xffffffffu, acc.re, o);
    acc.im += __shfl_down_sync(0xffffffffu, acc.im, o);
  }
  if (lane == 0) stc(y, (size_t)rhs * N + warp, acc);
}

int launch_dense_matvec(int pin, int pout, int N, const double2* inv, const void* x, void* y, int nrhs,
                        cudaStream_t st) {
  dim3 grid((N * 32 + 255) / 256, nrhs);
  if (pin == 0 && pout == 0)
    dense_matvec_kernel<double2, double2><<<grid, 256, 0, st>>>(N, inv, (const double2*)x, (double2*)y);
  else if (pin == 1 && pout == 1)
    dense_matvec_kernel<float2, float2><<<grid, 256, 0, st>>>(N, inv, (const float2*)x, (float2*)y);
  else
    return -1;
  return launched() ? 0 : -1;
}

}  // namespace wmg
