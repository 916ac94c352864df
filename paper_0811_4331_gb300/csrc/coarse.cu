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

static inline bool launched() { return launch_ok(); }

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
  const double* shift;  // null, or a diagonal shift per right-hand side
};

// G lanes cooperate on one output (i, B): lane q of the group sums the
// (d, j) terms q, q + G, ...; the group then reduces with shuffles.  Small
// coarse grids use large G so that the launch still covers every SM.
template <typename S, int NT, int G>
__global__ void __launch_bounds__(NT) coarse_apply_kernel(const CoarseArgs<S> A) {
  typedef typename Store<S>::R R;
  const int V = A.V, n = A.n;
  const int t = blockIdx.x * NT + threadIdx.x;
  const int o = t / G, q = t % G;  // output index o = i V + B
  const int rhs = blockIdx.y;
  const size_t voff = (size_t)rhs * n * V;
  R red[3] = {(R)0, (R)0, (R)0};
  const bool live = o < n * V;
  cx<R> acc = zero<R>();
  int i = 0, B = 0;
  if (live) {
    i = o / V;
    B = o - i * V;
    int c[4];
    site_coords(B, A.L, c);
    const int terms = 9 * n;
    int d = q / n, j = q - (q / n) * n;
    int nb = (q < terms) ? neighbor(c, A.L, d) : 0;
    auto next = [&]() {
      j += G;
      while (j >= n) {
        j -= n;
        ++d;
        if (d < 9) nb = neighbor(c, A.L, d);
      }
    };
    int p = q;
    // four terms' loads in flight per lane (the sum keeps its order)
    for (; p + 3 * G < terms; p += 4 * G) {
      cx<R> cv[4], xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cv[u] = ldc<R>(A.C, (((size_t)(d * n + i) * n) + j) * V + B);
        xv[u] = ldc<R>(A.in, voff + (size_t)j * V + nb);
        next();
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = cfma(cv[u], xv[u], acc);
    }
    for (; p < terms; p += G) {
      acc = cfma(ldc<R>(A.C, (((size_t)(d * n + i) * n) + j) * V + B), ldc<R>(A.in, voff + (size_t)j * V + nb), acc);
      next();
    }
  }
  if (G > 1) {
#pragma unroll
    for (int w = G / 2; w > 0; w >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, w);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, w);
    }
  }
  if (live && q == 0) {
    const size_t oo = voff + (size_t)i * V + B;
    if (A.shift) acc = cfma(mk<R>((R)A.shift[rhs], (R)0), ldc<R>(A.in, oo), acc);
    cx<R> v = (R)A.a * acc;
    if (A.y) v = v + (R)A.c * ldc<R>(A.y, oo);
    stc(A.out, oo, v);
    if (A.z) {
      const cx<R> vs = as_stored<S>(v);
      const cx<R> dd = cmul_conj(vs, ldc<R>(A.z, oo));
      red[0] = dd.re;
      red[1] = dd.im;
      red[2] = norm2(vs);
    }
  }
  if (A.z) grid_reduce<3, NT, R>(red, A.red, rhs);
}

// Lanes per output: enough threads for ~64K in flight, at most 32.
static int coarse_group(int ncomp, int V) {
  const long outs = (long)ncomp * V;
  int G = 1;
  while (G < 32 && outs * G < 65536) G *= 2;
  return G;
}

int launch_coarse_apply(const CoarseCall& k, cudaStream_t st) {
  constexpr int NT = 128;
  const int V = k.L[0] * k.L[1] * k.L[2] * k.L[3];
  const int G = coarse_group(k.ncomp, V);
  dim3 grid((unsigned)(((long)k.ncomp * V * G + NT - 1) / NT), k.nrhs);
#define WMG_COARSE_G(S, GG) coarse_apply_kernel<S, NT, GG><<<grid, NT, 0, st>>>(A)
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
    A.shift = k.shift;                                       \
    switch (G) {                                             \
      case 1: WMG_COARSE_G(S, 1); break;                     \
      case 2: WMG_COARSE_G(S, 2); break;                     \
      case 4: WMG_COARSE_G(S, 4); break;                     \
      case 8: WMG_COARSE_G(S, 8); break;                     \
      case 16: WMG_COARSE_G(S, 16); break;                   \
      default: WMG_COARSE_G(S, 32); break;                   \
    }                                                        \
  }
  switch (k.prec) {
    case 0: WMG_COARSE(double2); break;
    case 1: WMG_COARSE(float2); break;
    case 2: WMG_COARSE(__half2); break;
    case 3: WMG_COARSE(__nv_bfloat162); break;
    default: return -1;
  }
#undef WMG_COARSE
#undef WMG_COARSE_G
  return launched() ? 0 : -1;
}

int coarse_blocks(int ncomp, int V) {
  return (int)(((long)ncomp * V * coarse_group(ncomp, V) + 127) / 128);
}

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
// (fine field of chunk g.q, see fidx_q)
// One CTA per (aggregate, group of NT/32 rows): small coarse grids still fill the GPU.
template <typename SI, typename SP, typename SO, int NT>
__global__ void __launch_bounds__(NT) restrict_kernel(const Agg g, const SP* P, const SI* in, SO* out) {
  typedef typename Store<SP>::R R;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* sm = (cx<R>*)smem_raw;  // [ncomp][bsites]
  const int ngroups = (2 * g.nv + NT / 32 - 1) / (NT / 32);
  const int B = blockIdx.x / ngroups, grp = blockIdx.x % ngroups, rhs = blockIdx.y;
  const int bs = g.bsites, nh = g.nhalf;
  const SI* vin = in + (size_t)rhs * g.ncomp * g.V;
  for (int e = threadIdx.x; e < g.ncomp * bs; e += NT) {
    const int c = e / bs, s = e - c * bs;
    sm[e] = ldc<R>(vin, fidx_q(c, agg_site(g, B, s), g.V, g.q));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int len = nh * bs;
  {
    const int row = grp * (NT / 32) + warp;
    if (row >= 2 * g.nv) return;
    const int chi = row / g.nv;
    const SP* pr = P + ((size_t)B * 2 * g.nv + row) * len;
    const cx<R>* v = sm + (size_t)chi * len;
    cx<R> acc = zero<R>();
    int e = lane;
    // eight loads of P in flight per lane (the sum keeps its order)
    for (; e + 7 * 32 < len; e += 8 * 32) {
      cx<R> pv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) pv[u] = ldc<R>(pr, e + u * 32);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc = cfma_conj(pv[u], v[e + u * 32], acc);
    }
    for (; e < len; e += 32) acc = cfma_conj(ldc<R>(pr, e), v[e], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.re += __shfl_down_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_down_sync(0xffffffffu, acc.im, o);
    }
    if (lane == 0) stc(out, ((size_t)rhs * 2 * g.nv + row) * g.Vc + B, acc);
  }
}

// x[(chi nhalf + c)][site(B, s)] = sum_k P[B][chi][k][c][s] x_c[(chi nv + k)][B]
// One CTA per (aggregate, group of NT outputs).
template <typename SI, typename SP, typename SO, int NT>
__global__ void __launch_bounds__(NT) prolong_kernel(const Agg g, const SP* P, const SI* in, SO* out) {
  typedef typename Store<SP>::R R;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* xc = (cx<R>*)smem_raw;  // [2 nv]
  const int ngroups = (g.ncomp * g.bsites + NT - 1) / NT;
  const int B = blockIdx.x / ngroups, grp = blockIdx.x % ngroups, rhs = blockIdx.y;
  const int bs = g.bsites, nh = g.nhalf, nv = g.nv;
  for (int q = threadIdx.x; q < 2 * nv; q += NT) xc[q] = ldc<R>(in, ((size_t)rhs * 2 * nv + q) * g.Vc + B);
  __syncthreads();
  const size_t len = (size_t)nh * bs;
  {
    const int e = grp * NT + threadIdx.x;
    if (e >= g.ncomp * bs) return;
    const int c = e / bs, s = e - c * bs;
    const int chi = c / nh, cl = c - chi * nh;
    const SP* pc = P + ((size_t)B * 2 + chi) * nv * len + (size_t)cl * bs + s;
    cx<R> acc = zero<R>();
    int k = 0;
    // four loads of P in flight per thread (the sum keeps its order)
    for (; k + 3 < nv; k += 4) {
      cx<R> pv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pv[u] = ldc<R>(pc, (size_t)(k + u) * len);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = cfma(pv[u], xc[chi * nv + k + u], acc);
    }
    for (; k < nv; ++k) acc = cfma(ldc<R>(pc, (size_t)k * len), xc[chi * nv + k], acc);
    stc(out, (size_t)rhs * g.ncomp * g.V + fidx_q(c, agg_site(g, B, s), g.V, g.q), acc);
  }
}

template <typename SI, typename SP, typename SO>
static int restrict_t(const Agg& g, const void* P, const void* in, void* out, int nrhs, cudaStream_t st) {
  typedef typename Store<SP>::R R;
  constexpr int NT = 256;
  const size_t sm = (size_t)g.ncomp * g.bsites * sizeof(cx<R>);
  if (sm > 200 * 1024) return -1;
  if (sm > 48 * 1024)
    allow_big_smem(restrict_kernel<SI, SP, SO, NT>);
  const int ngroups = (2 * g.nv + NT / 32 - 1) / (NT / 32);
  restrict_kernel<SI, SP, SO, NT>
      <<<dim3(g.Vc * ngroups, nrhs), NT, sm, st>>>(g, (const SP*)P, (const SI*)in, (SO*)out);
  return launched() ? 0 : -1;
}

template <typename SI, typename SP, typename SO>
static int prolong_t(const Agg& g, const void* P, const void* in, void* out, int nrhs, cudaStream_t st) {
  typedef typename Store<SP>::R R;
  constexpr int NT = 256;
  const size_t sm = (size_t)2 * g.nv * sizeof(cx<R>);
  const int ngroups = (g.ncomp * g.bsites + NT - 1) / NT;
  prolong_kernel<SI, SP, SO, NT>
      <<<dim3(g.Vc * ngroups, nrhs), NT, sm, st>>>(g, (const SP*)P, (const SI*)in, (SO*)out);
  return launched() ? 0 : -1;
}

// Supported (vector-in, P, vector-out) precision triples.
int launch_restrict(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                    cudaStream_t st, int variant) {
  // several right-hand sides with 16-bit vectors and P: tensor cores, P read once
  if ((pin == 2 || pin == 3) && pP == pin && (pout == 1 || pout == pin) && transfer_mma_ok(g, nrhs))
    return launch_restrict_mma(pin, pP, pout, g, P, in, out, nrhs, st, variant);
  if (pin == 0 && pP == 0 && pout == 0) return restrict_t<double2, double2, double2>(g, P, in, out, nrhs, st);
  if (pin == 1 && pP == 1 && pout == 1) return restrict_t<float2, float2, float2>(g, P, in, out, nrhs, st);
  if (pin == 2 && pP == 2 && pout == 1) return restrict_t<__half2, __half2, float2>(g, P, in, out, nrhs, st);
  if (pin == 3 && pP == 3 && pout == 1)
    return restrict_t<__nv_bfloat162, __nv_bfloat162, float2>(g, P, in, out, nrhs, st);
  if (pin == 2 && pP == 2 && pout == 2) return restrict_t<__half2, __half2, __half2>(g, P, in, out, nrhs, st);
  if (pin == 3 && pP == 3 && pout == 3)
    return restrict_t<__nv_bfloat162, __nv_bfloat162, __nv_bfloat162>(g, P, in, out, nrhs, st);
  return -1;
}

int launch_prolong(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                   cudaStream_t st, int variant) {
  if ((pP == 2 || pP == 3) && pout == pP && (pin == 1 || pin == pP) && transfer_mma_ok(g, nrhs))
    return launch_prolong_mma(pin, pP, pout, g, P, in, out, nrhs, st, variant);
  if (pin == 0 && pP == 0 && pout == 0) return prolong_t<double2, double2, double2>(g, P, in, out, nrhs, st);
  if (pin == 1 && pP == 1 && pout == 1) return prolong_t<float2, float2, float2>(g, P, in, out, nrhs, st);
  if (pin == 1 && pP == 2 && pout == 2) return prolong_t<float2, __half2, __half2>(g, P, in, out, nrhs, st);
  if (pin == 1 && pP == 3 && pout == 3)
    return prolong_t<float2, __nv_bfloat162, __nv_bfloat162>(g, P, in, out, nrhs, st);
  if (pin == 2 && pP == 2 && pout == 2) return prolong_t<__half2, __half2, __half2>(g, P, in, out, nrhs, st);
  if (pin == 3 && pP == 3 && pout == 3)
    return prolong_t<__nv_bfloat162, __nv_bfloat162, __nv_bfloat162>(g, P, in, out, nrhs, st);
  return -1;
}

// C[0][i][i][B] += delta for every row i and coarse site B.
__global__ void diag_shift_kernel(double2* C, int n, int V, double delta) {
  const size_t tot = (size_t)n * V;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / V, B = e % V;
    C[(i * n + i) * V + B].x += delta;
  }
}

int launch_diag_shift(double2* C, int n, int V, double delta, cudaStream_t st) {
  const size_t tot = (size_t)n * V;
  size_t b = (tot + 255) / 256;
  if (b > 4096) b = 4096;
  diag_shift_kernel<<<(unsigned)(b < 1 ? 1 : b), 256, 0, st>>>(C, n, V, delta);
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ coarsest: dense inverse
// Dense matrix of a stencil operator in the internal vector order
// (row i V + B, column j V + B'), written into the left half of an
// augmented [N][2N] array (element type T); with ncol = 2N the right half
// is set to the identity, with ncol = N it is left alone.
template <typename T>
__global__ void stencil_to_dense_kernel(const double2* C, int L0, int L1, int L2, int L3, int n, int ncol, T* aug) {
  const int L[4] = {L0, L1, L2, L3};
  const int V = L0 * L1 * L2 * L3;
  const int N = n * V;
  const size_t tot = (size_t)N * ncol;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / ncol), col = (int)(e % ncol);
    cx<double> v = zero<double>();
    if (col < N) {
      const int i = row / V, B = row % V, j = col / V, Bp = col % V;
      int c[4];
      site_coords(B, L, c);
      for (int d = 0; d < 9; ++d) {
        if (neighbor(c, L, d) != Bp) continue;
        const double2 a = C[((size_t)(d * n + i) * n + j) * V + B];
        v.re += a.x;
        v.im += a.y;
      }
    } else if (col - N == row) {
      v.re = 1.0;
    }
    stc(aug, (size_t)row * 2 * N + col, v);
  }
}

// Gauss-Jordan elimination with virtual partial pivoting: rows are never
// swapped and pivot rows are never scaled during the sweep.  Step k takes the
// unused row p_k with the largest |a_{i,k}| as pivot and subtracts
// (a_ik / a_{p_k,k}) times row p_k from every other row; afterwards row p_k of
// the left block is a_{p_k,k} e_k, so row k of the inverse is row p_k of the
// right block divided by a_{p_k,k}.  One launch per step: the launch for
// step k also snapshots column k+1 and finds the next pivot with a packed
// 64-bit atomicMax (|a|^2 as float bits above, ~row below: ties go to the
// smallest row, independently of scheduling).
__device__ __forceinline__ unsigned long long pivot_key(float mag2, int row) {
  return ((unsigned long long)__float_as_uint(mag2) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)row);
}
__device__ __forceinline__ int pivot_row(unsigned long long key) { return (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFu)); }

template <typename T>
__global__ void gj_init_kernel(const T* aug, int N, T* col0, unsigned long long* keys) {
  typedef typename Store<T>::R R;
  const size_t ld = 2 * (size_t)N;
  unsigned long long best = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const T v = aug[(size_t)i * ld];
    col0[i] = v;
    const cx<R> c = ldc<R>(&v, 0);
    const unsigned long long key = pivot_key((float)norm2(c), i);
    best = key > best ? key : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, best, o);
    best = other > best ? other : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(keys, best);
}

// grid = (ceil((2N - k) / 256), N, batch): block row = matrix row i, columns
// k .. 2N-1, blockIdx.z = the matrix of a batch (independent eliminations
// that share the launches).  Per matrix z: aug at aug0 + z N 2N, column
// snapshots cols0 + z 2N (current (k & 1), next), pivot keys keys0 + z (N+1),
// used-row flags used0 + z N, error flag err0 + z.
template <typename T>
__global__ void gj_step_kernel(T* aug0, int N, int k, T* cols0, int* used0, unsigned long long* keys0, int* err0) {
  typedef typename Store<T>::R R;
  const int z = blockIdx.z;
  T* aug = aug0 + (size_t)z * N * 2 * N;
  const T* colk = cols0 + (size_t)z * 2 * N + (size_t)(k & 1) * N;
  T* colnext = cols0 + (size_t)z * 2 * N + (size_t)((k + 1) & 1) * N;
  int* used = used0 + (size_t)z * N;
  unsigned long long* keys = keys0 + (size_t)z * (N + 1);
  int* err = err0 + z;
  if (*err) return;
  const int i = blockIdx.y;
  const int j = k + blockIdx.x * blockDim.x + threadIdx.x;
  const int ld = 2 * N;
  const int p = pivot_row(keys[k]);
  if (p < 0 || p >= N) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *err = 1;
    return;
  }
  const cx<R> piv = ldc<R>(colk, p);
  if (!(norm2(piv) > (R)0)) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *err = 1;
    return;
  }
  if (j >= ld) return;
  const size_t o = (size_t)i * ld + j;
  cx<R> v = ldc<R>(aug, o);
  if (i != p) {
    const R den = norm2(piv);
    const cx<R> f = ldc<R>(colk, i) * mk<R>(piv.re / den, -piv.im / den);
    v = (j == k) ? zero<R>() : v - f * ldc<R>(aug, (size_t)p * ld + j);
    stc(aug, o, v);
  }
  if (j == k + 1 && j < N) {
    stc(colnext, i, v);
    if (i != p && !used[i]) atomicMax(keys + k + 1, pivot_key((float)norm2(v), i));
  }
  if (i == p && j == k) used[p] = 1;
}

// inv[k][c] = aug[p_k][N + c] / aug[p_k][k]
template <typename T>
__global__ void gj_finish_kernel(const T* aug, int N, const unsigned long long* keys, T* inv) {
  typedef typename Store<T>::R R;
  const size_t tot = (size_t)N * N;
  const size_t ld = 2 * (size_t)N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / N);
    const size_t c = e % N;
    const int p = pivot_row(keys[k]);
    if (p < 0 || p >= N) continue;
    const cx<R> piv = ldc<R>(aug, (size_t)p * ld + k);
    const R den = norm2(piv);
    const cx<R> pinv = mk<R>(piv.re / den, -piv.im / den);
    stc(inv, e, ldc<R>(aug, (size_t)p * ld + N + c) * pinv);
  }
}

static unsigned grid_for(size_t tot, size_t cap) {
  size_t b = (tot + 255) / 256;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------------ blocked Gauss-Jordan
// The same elimination (partial pivoting on the largest |a_ik|, rows kept in
// place, every other row eliminated) grouped in two levels.  A group of
// steps acts on the columns it does not pivot on as one linear map
// C -> T C with T = prod_j (1 - l_j e_{p_j}^+) (l_j zero at p_j); T = 1 - X E^+
// for E = [e_{p_0} .. e_{p_m-1}], so
//     T C = C - E C_P + (T E) C_P,
// where C_P are the m pivot rows of C before the group: pivot rows take
// (T E) C_P, every other row adds it.  The per-element arithmetic differs
// from the column-by-column order only by rounding.
//
// Right half in pivot order.  T e_q = e_q for every row q that is not yet a
// pivot, so the right half [A | 1] -> [T A | T] only ever holds, besides
// untouched unit columns, the columns T e_{p_s} of the rows already used.
// Slot s (column N + s) keeps T e_{p_s}: it is first written when row p_s
// becomes the pivot of step s (as the column of T E for that step) and the
// unit columns are never stored.  At the end column k of the left half is
// a_k e_{p_k}, and row k of the inverse is row p_k of T over a_k:
//     inv[k][p_s] = aug[p_k][N + s] / a_k.
//
// Outer blocks of kGjW steps: the columns outside the block's own columns
// that still change, i.e. the left columns right of the block and the slots
// of the earlier blocks' pivots, are the contiguous range
// [kb0 + W, N + kb0); they take one rank-W update per block (a dense
// product, gjb_outer_update_kernel).  Inside a block, panels of b columns:
// one CTA per matrix runs a panel's b steps with the rows in registers
// (gjb_panel_kernel) and a small rank-b update (gjb_inner_update_kernel)
// brings the rest of the block's columns and the block's earlier slots
// along.
constexpr int kGjW = 64;     // steps per outer block (a multiple of every panel width)
constexpr int kGjbRows = 4;  // rows per CTA of the inner update (many CTAs: the update is short)

// Panel kernel: one CTA per matrix z (blockIdx.x), b <= B steps on columns
// kb .. kb + b - 1.  Thread t owns rows t + m nt (m < RPT) and keeps their
// panel values P and tracker values Tr (the rows of T E) in registers; bit m
// of `mine` says whether its m-th row is already a pivot (or beyond N).
// Each step: the largest |a_ij| over the unused rows (one key per warp, then
// every warp reduces the warp keys itself), the owner of the pivot row
// publishes that row's panel and tracker values to shared memory, and every
// other row takes its multiple of it.  used[i] = step + 1 of the step that
// made row i a pivot (0: not yet).  Writes the panel back (zero off its
// pivot rows), T E into slots kb .. kb + b - 1, the pivots' keys, and the
// pivot rows of the inner update's columns (ranges [c1, c1 + n1) and
// [c2, c2 + n2)) into prow [8][kGjPRow] (rows b .. 7 unused).
constexpr int kGjPRow = 2 * kGjW;

template <typename T, int B, int RPT, int NT>
__global__ void __launch_bounds__(NT) gjb_panel_kernel(T* aug0, int N, int kb, int b, int c1, int n1, int c2,
                                                       int n2, unsigned long long* keys0, int* used0, T* prow0,
                                                       int* err0) {
  typedef typename Store<T>::R R;
  constexpr int LT = B + 1;  // padded row of a warp's staging tile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ cx<R> pr_s[2 * B];  // the pivot row: panel values, then tracker values
  __shared__ unsigned long long wkey[32];
  const int z = blockIdx.x;
  T* aug = aug0 + (size_t)z * N * 2 * N;
  unsigned long long* keys = keys0 + (size_t)z * (N + 1);
  int* used = used0 + (size_t)z * N;
  T* prow = prow0 + (size_t)z * 8 * kGjPRow;
  int* err = err0 + z;
  const int nt = blockDim.x, t = threadIdx.x, warp = t >> 5, lane = t & 31, nw = nt >> 5;
  const size_t ld = 2 * (size_t)N;
  // the warp's 32 consecutive rows (thread t owns row t + m nt) pass through its tile
  // [32][LT], so that global memory is read and written a row segment at a time
  cx<R>* tile = (cx<R>*)smem_raw + (size_t)warp * 32 * LT;
  if (*err) return;
  auto warp_max = [&](unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, v, o);
      v = other > v ? other : v;
    }
    return v;
  };
  cx<R> P[RPT][B], Tr[RPT][B];
  unsigned mine = 0;
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    const int i = t + m * nt, r0 = i - lane;
    if (i >= N || used[i]) mine |= 1u << m;
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int e = q * 32 + lane, r = e / B, j = e - r * B;
      tile[r * LT + j] = (j < b && r0 + r < N) ? ldc<R>(aug, (size_t)(r0 + r) * ld + kb + j) : zero<R>();
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < B; ++j) {
      P[m][j] = tile[lane * LT + j];
      Tr[m][j] = zero<R>();
    }
    __syncwarp();
  }
  int piv[B];
#pragma unroll
  for (int j = 0; j < B; ++j) {
    piv[j] = -1;
    if (j >= b) break;
    unsigned long long best = 0;
#pragma unroll
    for (int m = 0; m < RPT; ++m)
      if (!((mine >> m) & 1u)) {
        const unsigned long long key = pivot_key((float)norm2(P[m][j]), t + m * nt);
        best = key > best ? key : best;
      }
    best = warp_max(best);
    if (lane == 0) wkey[warp] = best;
    __syncthreads();  // every warp's key (and the previous step's reads of pr_s) are complete
    const unsigned long long v = warp_max(lane < nw ? wkey[lane] : 0ull);
    const int p = v ? pivot_row(v) : -1;
    if (p < 0 || p >= N) {
      if (t == 0) *err = 1;
      return;  // the same decision in every thread
    }
    piv[j] = p;
    if (p % nt == t) {  // the owner: row p's values, with its tracker unit set
      const int mp = p / nt;
#pragma unroll
      for (int m = 0; m < RPT; ++m)
        if (m == mp) {
          Tr[m][j] = mk<R>((R)1, (R)0);
          mine |= 1u << m;
#pragma unroll
          for (int jj = 0; jj < B; ++jj) {
            pr_s[jj] = P[m][jj];
            pr_s[B + jj] = Tr[m][jj];
          }
        }
      keys[kb + j] = v;
      used[p] = kb + j + 1;
    }
    __syncthreads();  // the pivot row is published
    const cx<R> pv = pr_s[j];
    const R den = norm2(pv);
    if (!(den > (R)0)) {
      if (t == 0) *err = 1;
      return;
    }
    const cx<R> pinv = mk<R>(pv.re / den, -pv.im / den);
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const int i = t + m * nt;
      if (i >= N || i == p) continue;
      const cx<R> l = P[m][j] * pinv;
#pragma unroll
      for (int jj = 0; jj < B; ++jj) {
        if (jj > j) {
          if (jj < b) P[m][jj] = P[m][jj] - l * pr_s[jj];
        } else {
          Tr[m][jj] = Tr[m][jj] - l * pr_s[B + jj];
        }
      }
    }
  }
  // the panel back (its columns zero off their pivot rows) and T E into the step's slots
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    const int i = t + m * nt, r0 = i - lane;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
      for (int j = 0; j < B; ++j) tile[lane * LT + j] = half ? Tr[m][j] : (i == piv[j] ? P[m][j] : zero<R>());
      __syncwarp();
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int e = q * 32 + lane, r = e / B, j = e - r * B;
        if (j < b && r0 + r < N) stc(aug, (size_t)(r0 + r) * ld + (half ? N : 0) + kb + j, tile[r * LT + j]);
      }
      __syncwarp();
    }
  }
  // the pivot rows of the inner update's columns, before that update
  const int nc = n1 + n2;
  for (int e = t; e < b * nc; e += nt) {
    const int j = e / nc, c = e - j * nc;
    const int col = c < n1 ? c1 + c : c2 + (c - n1);
    int pj = piv[0];
#pragma unroll
    for (int jj = 1; jj < B; ++jj)
      if (jj == j) pj = piv[jj];
    prow[(size_t)j * kGjPRow + c] = aug[(size_t)pj * ld + col];
  }
}

// Inner update of the block's other columns after a panel at kb (b steps):
// column c of the ranges [c1, c1 + n1) and [c2, c2 + n2) (index c' < n1 + n2
// in prow), row i:  a = (i a pivot of the panel ? 0 : a) + sum_j TE[i][j] prow[j][c'],
// TE[i][j] = aug[i][N + kb + j].  grid = (column tiles, row groups of
// kGjbRows, batch): a thread keeps its column's b pivot-row values in
// registers for kGjbRows rows; the group's TE rows and pivot flags sit in
// shared memory.
template <typename T>
__global__ void __launch_bounds__(128) gjb_inner_update_kernel(T* aug0, int N, int kb, int b, int c1, int n1, int c2,
                                                               int n2, const unsigned long long* keys0,
                                                               const T* prow0, const int* err0) {
  typedef typename Store<T>::R R;
  __shared__ cx<R> tes[kGjbRows][8];
  __shared__ int isp[kGjbRows];
  const int z = blockIdx.z;
  if (err0[z]) return;
  T* aug = aug0 + (size_t)z * N * 2 * N;
  const unsigned long long* keys = keys0 + (size_t)z * (N + 1);
  const T* prow = prow0 + (size_t)z * 8 * kGjPRow;
  const size_t ld = 2 * (size_t)N;
  const int i0 = blockIdx.y * kGjbRows;
  for (int e = threadIdx.x; e < kGjbRows * 8; e += blockDim.x) {  // all 8 slots: unused ones must be 0, not NaN
    const int r = e / 8, j = e % 8;
    tes[r][j] = (i0 + r < N && j < b) ? ldc<R>(aug, (size_t)(i0 + r) * ld + N + kb + j) : zero<R>();
  }
  if (threadIdx.x < kGjbRows) {
    int piv = 0;
    for (int j = 0; j < b; ++j) piv |= pivot_row(keys[kb + j]) == i0 + (int)threadIdx.x;
    isp[threadIdx.x] = piv;
  }
  __syncthreads();
  const int cc = blockIdx.x * blockDim.x + threadIdx.x;
  if (cc >= n1 + n2) return;
  const int c = cc < n1 ? c1 + cc : c2 + (cc - n1);
  cx<R> pr[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) pr[j] = j < b ? ldc<R>(prow, (size_t)j * kGjPRow + cc) : zero<R>();
  const int rows = min(kGjbRows, N - i0);
  cx<R> av[kGjbRows];
#pragma unroll
  for (int r = 0; r < kGjbRows; ++r) av[r] = r < rows ? ldc<R>(aug, (size_t)(i0 + r) * ld + c) : zero<R>();
#pragma unroll
  for (int r = 0; r < kGjbRows; ++r) {
    if (r >= rows) break;
    cx<R> acc = zero<R>();
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j < b) acc = cfma(tes[r][j], pr[j], acc);
    stc(aug, (size_t)(i0 + r) * ld + c, isp[r] ? acc : av[r] + acc);
  }
}

// Pivot rows of an outer block (steps kb0 .. kb0 + W - 1) over the columns
// [kb0 + W, N + kb0) that its update changes: cp[j][c] = aug[p_{kb0+j}][kb0 + W + c]
// (row stride N), taken before the update overwrites them.
template <typename T>
__global__ void gjb_gather_kernel(const T* aug0, int N, int kb0, int W, const unsigned long long* keys0, T* cp0,
                                  const int* err0) {
  const int z = blockIdx.z;
  if (err0[z]) return;
  const T* aug = aug0 + (size_t)z * N * 2 * N;
  const unsigned long long* keys = keys0 + (size_t)z * (N + 1);
  T* cp = cp0 + (size_t)z * kGjW * N;
  const int j = blockIdx.y, nc = N - W;
  const int p = pivot_row(keys[kb0 + j]);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
    cp[(size_t)j * N + c] = aug[(size_t)p * 2 * N + kb0 + W + c];
}

// Outer update after the block's W steps: rows i < N, columns c of
// [kb0 + W, N + kb0):  a = (i a pivot of the block ? 0 : a) + sum_{j<W} TE[i][j] cp[j][c],
// TE[i][j] = aug[i][N + kb0 + j] (the block's slots).  A dense product of
// N x W by W x (N - W) per matrix: CTA = kGjTile x kGjTile outputs, 256
// threads of 4 x 4 outputs each, both operand tiles in shared memory
// (TE row-major and padded, cp column-contiguous), K = W <= kGjW.
constexpr int kGjTile = 64;

template <typename T>
__global__ void __launch_bounds__(256) gjb_outer_update_kernel(T* aug0, int N, int kb0, int W, const int* used0,
                                                               const T* cp0, const int* err0) {
  typedef typename Store<T>::R R;
  constexpr int LA = kGjW + 1;  // padded row of the TE tile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* As = (cx<R>*)smem_raw;      // [kGjTile][LA]   TE rows
  cx<R>* Bs = As + kGjTile * LA;     // [kGjW][kGjTile] cp columns
  const int z = blockIdx.z;
  if (err0[z]) return;
  T* aug = aug0 + (size_t)z * N * 2 * N;
  const int* used = used0 + (size_t)z * N;
  const T* cp = cp0 + (size_t)z * kGjW * N;
  const size_t ld = 2 * (size_t)N;
  const int nc = N - W, cbase = kb0 + W;
  const int r0 = blockIdx.y * kGjTile, q0 = blockIdx.x * kGjTile;
  for (int e = threadIdx.x; e < kGjTile * kGjW; e += blockDim.x) {
    const int r = e / kGjW, k = e - r * kGjW;  // consecutive threads: consecutive slots of one row
    As[r * LA + k] = (r0 + r < N && k < W) ? ldc<R>(aug, (size_t)(r0 + r) * ld + N + kb0 + k) : zero<R>();
  }
  for (int e = threadIdx.x; e < kGjW * kGjTile; e += blockDim.x) {
    const int k = e / kGjTile, q = e - k * kGjTile;
    Bs[k * kGjTile + q] = (k < W && q0 + q < nc) ? ldc<R>(cp, (size_t)k * N + q0 + q) : zero<R>();
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  cx<R> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = zero<R>();
#pragma unroll 4
  for (int k = 0; k < W; ++k) {
    cx<R> av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[(ty * 4 + a) * LA + k];
#pragma unroll
    for (int c = 0; c < 4; ++c) bv[c] = Bs[k * kGjTile + tx * 4 + c];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = cfma(av[a], bv[c], acc[a][c]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = r0 + ty * 4 + a;
    if (i >= N) break;
    const bool piv = (unsigned)(used[i] - 1 - kb0) < (unsigned)W;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int q = q0 + tx * 4 + c;
      if (q >= nc) break;
      const size_t o = (size_t)i * ld + cbase + q;
      stc(aug, o, piv ? acc[a][c] : ldc<R>(aug, o) + acc[a][c]);
    }
  }
}

// inv[k][p_s] = aug[p_k][N + s] / aug[p_k][k]   (the right half in pivot order)
template <typename T>
__global__ void gjb_finish_kernel(const T* aug, int N, const unsigned long long* keys, T* inv) {
  typedef typename Store<T>::R R;
  const size_t tot = (size_t)N * N;
  const size_t ld = 2 * (size_t)N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / N), s = (int)(e % N);
    const int p = pivot_row(keys[k]), ps = pivot_row(keys[s]);
    if (p < 0 || p >= N || ps < 0 || ps >= N) continue;
    const cx<R> piv = ldc<R>(aug, (size_t)p * ld + k);
    const R den = norm2(piv);
    const cx<R> pinv = mk<R>(piv.re / den, -piv.im / den);
    stc(inv, (size_t)k * N + ps, ldc<R>(aug, (size_t)p * ld + N + s) * pinv);
  }
}

// Panel shapes (width B, rows per thread RPT, threads NT), widest first: a
// thread's rows of the panel and its tracker sit in registers, so RPT x B is
// bounded by the register file (NT threads x the registers each needs).
struct GjbShape {
  int b, rpt, nt;
};
constexpr GjbShape kGjbF32[] = {{8, 1, 1024}, {8, 2, 640}, {8, 4, 384}, {4, 4, 640}, {4, 8, 384}, {2, 8, 640},
                                {2, 16, 384}};
constexpr GjbShape kGjbF64[] = {{8, 1, 512}, {4, 1, 1024}, {4, 2, 640}, {4, 4, 384}, {2, 4, 640}, {2, 8, 384}};

// The first shape whose threads x rows cover N; b = 0: none (single steps).
static GjbShape gjb_shape(int N, size_t eb) {
  const GjbShape* s = eb == 8 ? kGjbF32 : kGjbF64;
  const int n = eb == 8 ? (int)(sizeof(kGjbF32) / sizeof(GjbShape)) : (int)(sizeof(kGjbF64) / sizeof(GjbShape));
  for (int k = 0; k < n; ++k)
    if ((long long)s[k].nt * s[k].rpt >= N) return s[k];
  return GjbShape{0, 0, 0};
}

size_t gjb_scratch_bytes(int N, size_t eb, int batch) {
  const int b = gjb_shape(N, eb).b;
  return b ? (size_t)batch * ((size_t)8 * kGjPRow + (size_t)kGjW * N) * eb + 256 : 0;
}

template <typename T>
using GjbPanel = void (*)(T*, int, int, int, int, int, int, int, unsigned long long*, int*, T*, int*);

template <typename T>
static GjbPanel<T> gjb_panel_for(const GjbShape& s) {
  if constexpr (sizeof(T) == 8) {
    if (s.b == 8 && s.rpt == 1) return gjb_panel_kernel<T, 8, 1, 1024>;
    if (s.b == 8 && s.rpt == 2) return gjb_panel_kernel<T, 8, 2, 640>;
    if (s.b == 8 && s.rpt == 4) return gjb_panel_kernel<T, 8, 4, 384>;
    if (s.b == 4 && s.rpt == 4) return gjb_panel_kernel<T, 4, 4, 640>;
    if (s.b == 4 && s.rpt == 8) return gjb_panel_kernel<T, 4, 8, 384>;
    if (s.b == 2 && s.rpt == 8) return gjb_panel_kernel<T, 2, 8, 640>;
    return gjb_panel_kernel<T, 2, 16, 384>;
  } else {
    if (s.b == 8 && s.rpt == 1) return gjb_panel_kernel<T, 8, 1, 512>;
    if (s.b == 4 && s.rpt == 1) return gjb_panel_kernel<T, 4, 1, 1024>;
    if (s.b == 4 && s.rpt == 2) return gjb_panel_kernel<T, 4, 2, 640>;
    if (s.b == 4 && s.rpt == 4) return gjb_panel_kernel<T, 4, 4, 384>;
    if (s.b == 2 && s.rpt == 4) return gjb_panel_kernel<T, 2, 4, 640>;
    return gjb_panel_kernel<T, 2, 8, 384>;
  }
}

template <typename T>
static int dense_inverse_t(const double2* const* C, const int L[4], int n, int batch, T* aug, char* sc, int* err,
                           void* const* inv, void* blk, cudaStream_t st, long long* launches) {
  const int V = L[0] * L[1] * L[2] * L[3];
  const int N = n * V;
  const size_t nn2 = (size_t)N * 2 * N;
  T* cols = (T*)sc;
  unsigned long long* keys = (unsigned long long*)(sc + (size_t)batch * 2 * N * sizeof(T));
  int* used = (int*)(keys + (size_t)batch * (N + 1));
  long long nl = 0;
  cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (N + 1) * batch, st);
  cudaMemsetAsync(used, 0, sizeof(int) * N * batch, st);
  const GjbShape shape = blk ? gjb_shape(N, sizeof(T)) : GjbShape{0, 0, 0};
  const int b = shape.b;
  for (int z = 0; z < batch; ++z) {
    // the blocked form never reads a unit column of the right half (slots are written when used)
    const int ncol = b ? N : 2 * N;
    stencil_to_dense_kernel<T><<<grid_for((size_t)N * ncol, 8192), 256, 0, st>>>(C[z], L[0], L[1], L[2], L[3], n,
                                                                                 ncol, aug + z * nn2);
    ++nl;
    if (!b) {
      gj_init_kernel<T><<<grid_for(N, 1024), 256, 0, st>>>(aug + z * nn2, N, cols + (size_t)z * 2 * N,
                                                           keys + (size_t)z * (N + 1));
      ++nl;
    }
  }
  if (!launched()) return -1;
  if (b) {
    T* prow = (T*)blk;
    T* cp = prow + (size_t)batch * 8 * kGjPRow;
    const int pnt = ((N + shape.rpt - 1) / shape.rpt + 31) / 32 * 32;  // threads of a panel CTA
    const size_t psm = (size_t)(pnt / 32) * 32 * (shape.b + 1) * sizeof(T);  // the warps' staging tiles
    auto panel = gjb_panel_for<T>(shape);
    allow_big_smem(panel);
    const size_t smo = ((size_t)kGjTile * (kGjW + 1) + (size_t)kGjW * kGjTile) * sizeof(T);
    allow_big_smem(gjb_outer_update_kernel<T>);
    for (int kb0 = 0; kb0 < N; kb0 += kGjW) {
      const int W = N - kb0 < kGjW ? N - kb0 : kGjW;
      for (int kb = kb0; kb < kb0 + W; kb += b) {
        const int bw = kb0 + W - kb < b ? kb0 + W - kb : b;
        // the block's columns right of the panel, and the block's earlier slots
        const int c1 = kb + bw, n1 = kb0 + W - c1, c2 = N + kb0, n2 = kb - kb0;
        panel<<<batch, pnt, psm, st>>>(aug, N, kb, bw, c1, n1, c2, n2, keys, used, prow, err);
        ++nl;
        if (n1 + n2 > 0) {
          const dim3 grid((unsigned)((n1 + n2 + 127) / 128), (unsigned)((N + kGjbRows - 1) / kGjbRows),
                          (unsigned)batch);
          gjb_inner_update_kernel<T><<<grid, 128, 0, st>>>(aug, N, kb, bw, c1, n1, c2, n2, keys, prow, err);
          ++nl;
        }
      }
      if (N - W > 0) {
        const dim3 gg((unsigned)((N - W + 255) / 256 < 16 ? (N - W + 255) / 256 : 16), (unsigned)W, (unsigned)batch);
        gjb_gather_kernel<T><<<gg, 256, 0, st>>>(aug, N, kb0, W, keys, cp, err);
        const dim3 go((unsigned)((N - W + kGjTile - 1) / kGjTile), (unsigned)((N + kGjTile - 1) / kGjTile),
                      (unsigned)batch);
        gjb_outer_update_kernel<T><<<go, 256, smo, st>>>(aug, N, kb0, W, used, cp, err);
        nl += 2;
      }
    }
    for (int z = 0; z < batch; ++z)
      gjb_finish_kernel<T><<<grid_for((size_t)N * N, 8192), 256, 0, st>>>(aug + z * nn2, N, keys + (size_t)z * (N + 1),
                                                                          (T*)inv[z]);
  } else {
    for (int k = 0; k < N; ++k) {
      const dim3 grid((unsigned)((2 * N - k + 255) / 256), (unsigned)N, (unsigned)batch);
      gj_step_kernel<T><<<grid, 256, 0, st>>>(aug, N, k, cols, used, keys, err);
    }
    nl += N;
    for (int z = 0; z < batch; ++z)
      gj_finish_kernel<T><<<grid_for((size_t)N * N, 8192), 256, 0, st>>>(aug + z * nn2, N, keys + (size_t)z * (N + 1),
                                                                        (T*)inv[z]);
  }
  nl += batch;
  if (launches) *launches = nl;
  return launched() ? 0 : -1;
}

int dense_inverse_batch(int prec, const double2* const* C, const int L[4], int n, int batch, void* aug, void* scratch,
                        int* err, void* const* inv, void* blk, cudaStream_t st, long long* launches) {
  // scratch: per matrix two column snapshots [2][N] of the element type, then N + 1 pivot keys per
  // matrix, then N pivot-step flags per matrix; blk (optional): the blocked form's pivot rows
  if (batch < 1) return -1;
  if (prec == 0)
    return dense_inverse_t<double2>(C, L, n, batch, (double2*)aug, (char*)scratch, err, inv, blk, st, launches);
  if (prec == 1)
    return dense_inverse_t<float2>(C, L, n, batch, (float2*)aug, (char*)scratch, err, inv, blk, st, launches);
  return -1;
}

int dense_inverse(int prec, const double2* C, const int L[4], int n, void* aug, void* scratch, int* err, void* inv,
                  cudaStream_t st) {
  void* invs[1] = {inv};
  return dense_inverse_batch(prec, &C, L, n, 1, aug, scratch, err, invs, nullptr, st, nullptr);
}

size_t dense_inverse_scratch_bytes(int prec, int N) {
  return 2 * (size_t)N * (prec == 0 ? 16 : 8) + 8 * ((size_t)N + 1) + 4 * (size_t)N + 64;
}

// Y = inv X (+ Y if acc) for 4 <= nrhs <= 64: a dense product, tiled so that
// each element of the inverse is read once per launch instead of once per
// right-hand side.  CTA (tile, ks) owns 16 rows, every right-hand side and the
// ks-th of KS contiguous K ranges; a K step stages 16 x 32 of the inverse and
// 32 x nrhs of X in shared memory; thread t accumulates row t % 16 for the
// right-hand sides t / 16 + 16 q.  The K ranges keep the dependent chain of
// each CTA short enough to fill the GPU (the coarsest matrix has ~1500 rows).
// Each CTA parks its partial tile; the last CTA of a row tile to finish (an
// atomic ticket, reset by it) adds the KS partials in ks order and writes Y,
// so the sum is deterministic.  Arithmetic in the matrix's precision.
constexpr int kMmRows = 16, kMmK = 32, kMmThreads = 256;

template <typename TM, typename SI, typename SO>
__global__ void __launch_bounds__(kMmThreads)
    dense_matmul_kernel(int N, const TM* inv, const SI* x, SO* y, int R, int acc, int kper,
                        cx<typename Store<TM>::R>* part, unsigned* tickets) {
  typedef typename Store<TM>::R Rt;
  __shared__ cx<Rt> As[kMmRows][kMmK + 1];
  __shared__ cx<Rt> Bs[kMmK][64];
  __shared__ unsigned last;
  const int row0 = blockIdx.x * kMmRows, ks = blockIdx.y, KS = gridDim.y;
  const int kbeg = ks * kper, kend = min(N, kbeg + kper);
  const int tr = threadIdx.x % kMmRows, tg = threadIdx.x / kMmRows;  // row in tile, rhs group (0..15)
  constexpr int kPer = 4;                                             // 64 rhs / 16 groups
  cx<Rt> accv[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) accv[q] = zero<Rt>();
  for (int k0 = kbeg; k0 < kend; k0 += kMmK) {
    for (int e = threadIdx.x; e < kMmRows * kMmK; e += kMmThreads) {
      const int r = e / kMmK, c = e % kMmK;
      const int gr = row0 + r, gc = k0 + c;
      As[r][c] = (gr < N && gc < kend) ? ldc<Rt>(inv, (size_t)gr * N + gc) : zero<Rt>();
    }
    for (int e = threadIdx.x; e < kMmK * R; e += kMmThreads) {
      const int r = e / kMmK, c = e % kMmK;
      Bs[c][r] = (k0 + c < kend) ? ldc<Rt>(x, (size_t)r * N + k0 + c) : zero<Rt>();
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kMmK; ++kk) {
      const cx<Rt> a = As[tr][kk];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int r = tg + 16 * q;
        if (r < R) accv[q] = cfma(a, Bs[kk][r], accv[q]);
      }
    }
    __syncthreads();
  }
  const int grow = row0 + tr;
  // park this K range's tile: part[ks][r][row]
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int r = tg + 16 * q;
    if (r < R && grow < N) part[((size_t)ks * R + r) * N + grow] = accv[q];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&tickets[blockIdx.x], 1u) == (unsigned)(KS - 1));
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (grow < N) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int r = tg + 16 * q;
      if (r >= R) break;
      const volatile Rt* pv = (const volatile Rt*)part;  // other CTAs' tiles, past the ticket
      cx<Rt> sum = zero<Rt>();
      for (int j = 0; j < KS; ++j) {
        const size_t idx = ((size_t)j * R + r) * N + grow;
        sum = sum + mk<Rt>(pv[2 * idx], pv[2 * idx + 1]);
      }
      const size_t o = (size_t)r * N + grow;
      cx<double> v = mk<double>((double)sum.re, (double)sum.im);
      if (acc) v = v + ldc<double>(y, o);
      stc(y, o, v);
    }
  }
  if (threadIdx.x == 0) tickets[blockIdx.x] = 0u;
}

// Scratch of the tiled product: partial tiles (up to 8 K ranges x 64 rhs x N
// complex FP64) and one ticket per 16-row tile.
size_t dense_matvec_scratch_bytes(int N) {
  return (size_t)8 * 64 * N * 16 + (size_t)((N + kMmRows - 1) / kMmRows) * sizeof(unsigned) + 256;
}

// y = inv x (+ y if acc) for 1-3 right-hand sides: a CTA of kMvWarps warps per
// row, warp w summing columns [w N / kMvWarps, (w+1) N / kMvWarps) with two
// independent chains, the warps' sums added in warp order (deterministic).
constexpr int kMvWarps = 4;

template <typename TM, typename SI, typename SO>
__global__ void __launch_bounds__(32 * kMvWarps) dense_matvec4_kernel(int N, const TM* inv, const SI* x, SO* y,
                                                                      int acc, const int* midx) {
  typedef typename Store<TM>::R R;
  __shared__ cx<R> part[kMvWarps];
  const int row = blockIdx.x, rhs = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = (int)((long)warp * N / kMvWarps), c1 = (int)((long)(warp + 1) * N / kMvWarps);
  const TM* rp = inv + (midx ? (size_t)midx[rhs] * N * N : (size_t)0) + (size_t)row * N;
  const SI* xr = x + (size_t)rhs * N;
  cx<R> a = zero<R>(), b = zero<R>();
  int j = c0 + lane;
  // eight loads in flight per lane; chain a takes columns j, j + 64, ..., chain b j + 32, j + 96, ...
  for (; j + 96 < c1; j += 128) {
    const cx<R> m0 = ldc<R>(rp, j), m1 = ldc<R>(rp, j + 32), m2 = ldc<R>(rp, j + 64), m3 = ldc<R>(rp, j + 96);
    const cx<R> x0 = ldc<R>(xr, j), x1 = ldc<R>(xr, j + 32), x2 = ldc<R>(xr, j + 64), x3 = ldc<R>(xr, j + 96);
    a = cfma(m0, x0, a);
    b = cfma(m1, x1, b);
    a = cfma(m2, x2, a);
    b = cfma(m3, x3, b);
  }
  for (; j + 32 < c1; j += 64) {
    a = cfma(ldc<R>(rp, j), ldc<R>(xr, j), a);
    b = cfma(ldc<R>(rp, j + 32), ldc<R>(xr, j + 32), b);
  }
  for (; j < c1; j += 32) a = cfma(ldc<R>(rp, j), ldc<R>(xr, j), a);
  a = a + b;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a.re += __shfl_down_sync(0xffffffffu, a.re, o);
    a.im += __shfl_down_sync(0xffffffffu, a.im, o);
  }
  if (lane == 0) part[warp] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    cx<R> s = part[0];
#pragma unroll
    for (int w = 1; w < kMvWarps; ++w) s = s + part[w];
    const size_t o = (size_t)rhs * N + row;
    cx<double> v = mk<double>((double)s.re, (double)s.im);
    if (acc) v = v + ldc<double>(y, o);
    stc(y, o, v);
  }
}

int launch_dense_matvec(int pm, int pin, int pout, int N, const void* inv, const void* x, void* y, int nrhs, int acc,
                        cudaStream_t st, void* scratch, const int* midx) {
  if (nrhs < 4 || !scratch || midx) {
    const dim3 g((unsigned)N, (unsigned)nrhs);
    if (pm == 0 && pin == 0 && pout == 0)
      dense_matvec4_kernel<double2, double2, double2>
          <<<g, 32 * kMvWarps, 0, st>>>(N, (const double2*)inv, (const double2*)x, (double2*)y, acc, midx);
    else if (pm == 1 && pin == 0 && pout == 0)
      dense_matvec4_kernel<float2, double2, double2>
          <<<g, 32 * kMvWarps, 0, st>>>(N, (const float2*)inv, (const double2*)x, (double2*)y, acc, midx);
    else if (pm == 1 && pin == 1 && pout == 1)
      dense_matvec4_kernel<float2, float2, float2>
          <<<g, 32 * kMvWarps, 0, st>>>(N, (const float2*)inv, (const float2*)x, (float2*)y, acc, midx);
    else
      return -1;
    return launched() ? 0 : -1;
  }
  if (scratch && nrhs >= 4 && nrhs <= 64) {
    const int tiles = (N + kMmRows - 1) / kMmRows;
    int KS = (2 * sm_count() + tiles - 1) / tiles;  // about two CTAs per SM
    KS = KS < 1 ? 1 : (KS > 8 ? 8 : KS);
    int kper = (N + KS - 1) / KS;
    kper = (kper + kMmK - 1) / kMmK * kMmK;
    KS = (N + kper - 1) / kper;
    const dim3 g(tiles, KS);
    unsigned* tickets = (unsigned*)((char*)scratch + (size_t)8 * 64 * N * 16);
    if (pm == 0 && pin == 0 && pout == 0)
      dense_matmul_kernel<double2, double2, double2><<<g, kMmThreads, 0, st>>>(
          N, (const double2*)inv, (const double2*)x, (double2*)y, nrhs, acc, kper, (cx<double>*)scratch, tickets);
    else if (pm == 1 && pin == 0 && pout == 0)
      dense_matmul_kernel<float2, double2, double2><<<g, kMmThreads, 0, st>>>(
          N, (const float2*)inv, (const double2*)x, (double2*)y, nrhs, acc, kper, (cx<float>*)scratch, tickets);
    else if (pm == 1 && pin == 1 && pout == 1)
      dense_matmul_kernel<float2, float2, float2><<<g, kMmThreads, 0, st>>>(
          N, (const float2*)inv, (const float2*)x, (float2*)y, nrhs, acc, kper, (cx<float>*)scratch, tickets);
    else
      return -1;
    return launched() ? 0 : -1;
  }
  return -1;
}

}  // namespace wmg
