// Vector kernels of the solver: MR and alpha-step updates (Sec. 3), GCR
// Gram-Schmidt and updates (Sec. 5), precision conversion, layout transposes
// and the counter-based start vectors of the null-vector setup (Sec. 2).
//
// All reductions are deterministic (a grid fixed by the vector length and the
// device's SM count, last-block finish, see grid_reduce).  The FP64 kernels
// accumulate in FP64; the FP32 and 16-bit kernels accumulate per thread and
// within a block in FP32 and sum the per-block partials in FP64.  Grids are
// capped at 8 blocks per SM (at most kMaxVecBlocks) with grid-stride loops, so
// every vector kernel is one coalesced streaming pass over its operands.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace wmg {

int vec_blocks(size_t n) {
  size_t b = (n + kVecThreads - 1) / kVecThreads;
  const size_t cap = (size_t)8 * sm_count() < (size_t)kMaxVecBlocks ? (size_t)8 * sm_count() : (size_t)kMaxVecBlocks;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

static inline bool launched() { return launch_ok(); }

// Blocks of the dot kernels: at least 8 elements per thread, at most one block per SM.
int red_blocks(size_t n) {
  size_t b = (n + 8 * kVecThreads - 1) / (8 * kVecThreads);
  const size_t cap = (size_t)sm_count() < (size_t)kMaxVecBlocks ? (size_t)sm_count() : (size_t)kMaxVecBlocks;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------------ MR update
// Per-right-hand-side scalars are formed once per CTA by its first thread (in
// FP64, from the FP64 reduction slots) and shared: FP64 division and square
// root run at a small fraction of the FP32 rate on this part, so no thread of
// a vector kernel evaluates them for itself.
template <typename R>
__device__ __forceinline__ cx<R> mr_alpha(const MrUpdate& m, int rhs) {
  __shared__ double sa[2];
  if (threadIdx.x == 0) {
    const double* d = m.dots + (size_t)rhs * m.dstride;
    const double den = d[2];
    double ar = 0.0, ai = 0.0;
    if (den > 0.0 && isfinite(den)) {
      ar = m.omega * d[0] / den;
      ai = m.omega * d[1] / den;
    }
    sa[0] = ar;
    sa[1] = ai;
  }
  __syncthreads();
  return mk<R>((R)sa[0], (R)sa[1]);
}

template <typename S>
__global__ void __launch_bounds__(kVecThreads) mr_update_kernel(const MrUpdate m) {
  typedef typename Store<S>::R R;
  const int rhs = blockIdx.y;
  const cx<R> alpha = mr_alpha<R>(m, rhs);
  const size_t off = (size_t)rhs * m.n;
  S* xo = (S*)m.x_out + off;
  const S* xi = m.x_in ? (const S*)m.x_in + off : nullptr;
  const S* u = (const S*)m.u + off;
  S* ro = (S*)m.r_out + off;
  const S* ri = (const S*)m.r_in + off;
  const S* p = (const S*)m.p + off;
  R acc = (R)0;  // per-thread partial in the arithmetic type; FP64 only across threads
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < m.n; i += (size_t)gridDim.x * kVecThreads) {
    cx<R> x = xi ? ldc<R>(xi, i) : zero<R>();
    x = cfma(alpha, ldc<R>(u, i), x);
    cx<R> r = ldc<R>(ri, i);
    r = r - alpha * ldc<R>(p, i);
    stc(xo, i, x);
    stc(ro, i, r);
    acc += norm2(as_stored<S>(r));
  }
  R red[1] = {acc};
  if (m.red.result) grid_reduce<1, kVecThreads, R>(red, m.red, rhs);
}

// 16-bit storage: a thread moves two complex numbers per access (8-byte
// loads and stores instead of 4-byte ones; the per-element work is the same).
template <typename S>
struct __align__(8) Pair16 {
  S a, b;
};

template <typename S>
__global__ void __launch_bounds__(kVecThreads) mr_update2_kernel(const MrUpdate m) {
  typedef Pair16<S> P2;
  const int rhs = blockIdx.y;
  const cx<float> alpha = mr_alpha<float>(m, rhs);
  const size_t off = (size_t)rhs * m.n / 2;
  P2* xo = (P2*)m.x_out + off;
  const P2* xi = m.x_in ? (const P2*)m.x_in + off : nullptr;
  const P2* u = (const P2*)m.u + off;
  P2* ro = (P2*)m.r_out + off;
  const P2* ri = (const P2*)m.r_in + off;
  const P2* p = (const P2*)m.p + off;
  const unsigned n2 = (unsigned)(m.n / 2);
  float acc = 0.f;
  for (unsigned i = blockIdx.x * kVecThreads + threadIdx.x; i < n2; i += gridDim.x * kVecThreads) {
    const P2 uu = u[i], rr = ri[i], pp = p[i];
    P2 xx;
    if (xi) xx = xi[i];
    cx<float> x0 = xi ? ldc<float>(&xx.a, 0) : zero<float>(), x1 = xi ? ldc<float>(&xx.b, 0) : zero<float>();
    x0 = cfma(alpha, ldc<float>(&uu.a, 0), x0);
    x1 = cfma(alpha, ldc<float>(&uu.b, 0), x1);
    const cx<float> r0 = ldc<float>(&rr.a, 0) - alpha * ldc<float>(&pp.a, 0);
    const cx<float> r1 = ldc<float>(&rr.b, 0) - alpha * ldc<float>(&pp.b, 0);
    P2 xw, rw;
    stc(&xw.a, 0, x0);
    stc(&xw.b, 0, x1);
    stc(&rw.a, 0, r0);
    stc(&rw.b, 0, r1);
    xo[i] = xw;
    ro[i] = rw;
    acc += norm2(as_stored<S>(r0)) + norm2(as_stored<S>(r1));
  }
  float red[1] = {acc};
  if (m.red.result) grid_reduce<1, kVecThreads, float>(red, m.red, rhs);
}

int launch_mr_update(const MrUpdate& m, cudaStream_t st) {
  dim3 grid(vec_blocks(m.n), m.nrhs);
  auto al8 = [](const void* q) { return ((uintptr_t)q & 7u) == 0; };
  const bool pairs = (m.prec == 2 || m.prec == 3) && m.n % 2 == 0 && m.n / 2 < (1u << 31) && al8(m.x_out) &&
                     al8(m.x_in) && al8(m.u) && al8(m.r_out) && al8(m.r_in) && al8(m.p);
  if (pairs) grid.x = vec_blocks(m.n / 2);
  switch (m.prec) {
    case 0: mr_update_kernel<double2><<<grid, kVecThreads, 0, st>>>(m); break;
    case 1: mr_update_kernel<float2><<<grid, kVecThreads, 0, st>>>(m); break;
    case 2:
      if (pairs)
        mr_update2_kernel<__half2><<<grid, kVecThreads, 0, st>>>(m);
      else
        mr_update_kernel<__half2><<<grid, kVecThreads, 0, st>>>(m);
      break;
    case 3:
      if (pairs)
        mr_update2_kernel<__nv_bfloat162><<<grid, kVecThreads, 0, st>>>(m);
      else
        mr_update_kernel<__nv_bfloat162><<<grid, kVecThreads, 0, st>>>(m);
      break;
    default: return -1;
  }
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ dot
template <typename S>
__global__ void __launch_bounds__(kVecThreads) dot_kernel(size_t n, const S* a, const S* b, RedArgs ra) {
  typedef typename Store<S>::R R;
  const int rhs = blockIdx.y;
  a += (size_t)rhs * n;
  b += (size_t)rhs * n;
  R acc[4] = {(R)0, (R)0, (R)0, (R)0};
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecThreads) {
    cx<R> x = ldc<R>(a, i), y = ldc<R>(b, i);
    cx<R> d = cmul_conj(x, y);
    acc[0] += d.re;
    acc[1] += d.im;
    acc[2] += norm2(x);
    acc[3] += norm2(y);
  }
  grid_reduce<4, kVecThreads, R>(acc, ra, rhs);
}

int launch_dot(int prec, size_t n, int nrhs, const void* a, const void* b, RedArgs red, cudaStream_t st) {
  dim3 grid(red_blocks(n), nrhs);
  switch (prec) {
    case 0: dot_kernel<double2><<<grid, kVecThreads, 0, st>>>(n, (const double2*)a, (const double2*)b, red); break;
    case 1: dot_kernel<float2><<<grid, kVecThreads, 0, st>>>(n, (const float2*)a, (const float2*)b, red); break;
    case 2: dot_kernel<__half2><<<grid, kVecThreads, 0, st>>>(n, (const __half2*)a, (const __half2*)b, red); break;
    case 3:
      dot_kernel<__nv_bfloat162>
          <<<grid, kVecThreads, 0, st>>>(n, (const __nv_bfloat162*)a, (const __nv_bfloat162*)b, red);
      break;
    default: return -1;
  }
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ GCR Gram-Schmidt
// One block row computes CH dots <W_j|w> for j in [chunk * CH, chunk * CH + CH).
constexpr int kChunk = 8;

// The basis holds a multiple of kChunk vectors, so every block reads all
// kChunk vectors of its chunk without a bound test (the dots beyond k are
// computed from whatever the unused slots hold and are never read), and the
// eight loads of an element issue back to back.
// Second Gram-Schmidt pass on demand: with `pre` and `post` (the squared norm
// of w before and after the first pass, `cstride` doubles between right-hand
// sides) a pass runs for a right-hand side only where the first one removed
// more than half of ||w||^2 -- the reorthogonalisation test of Daniel,
// Gragg, Kaufman and Stewart (Math. Comp. 30, 1976) with eta = 1/sqrt(2).
// Every block of a right-hand side takes the same decision before it touches
// a reduction, so a skipped right-hand side leaves its tickets and slots as
// they were.
__device__ __forceinline__ bool gs_pass_skipped(const double* pre, const double* post, int cstride, int rhs) {
  if (!pre) return false;
  return !(post[(size_t)rhs * cstride] < 0.5 * pre[(size_t)rhs * cstride]);
}

template <typename S>
__global__ void __launch_bounds__(kVecThreads)
    multidot_kernel(size_t n, int k, int kmax, const S* W, size_t jstride, const S* w, RedArgs ra,
                    const double* pre, const double* post, int cstride) {
  typedef typename Store<S>::R R;
  const int chunk = blockIdx.y, rhs = blockIdx.z;
  if (gs_pass_skipped(pre, post, cstride, rhs)) return;
  const int j0 = chunk * kChunk;
  const S* wr = w + (size_t)rhs * n;
  const S* Wc = W + (size_t)j0 * jstride + (size_t)rhs * n;
  cx<R> acc[kChunk];
#pragma unroll
  for (int q = 0; q < kChunk; ++q) acc[q] = zero<R>();
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecThreads) {
    const cx<R> x = ldc<R>(wr, i);
    cx<R> v[kChunk];
#pragma unroll
    for (int q = 0; q < kChunk; ++q) v[q] = ldc<R>(Wc + (size_t)q * jstride, i);
#pragma unroll
    for (int q = 0; q < kChunk; ++q) acc[q] = cfma_conj(v[q], x, acc[q]);
  }
  R red[2 * kChunk];
#pragma unroll
  for (int q = 0; q < kChunk; ++q) {
    red[2 * q] = acc[q].re;
    red[2 * q + 1] = acc[q].im;
  }
  // lane = rhs * nchunks + chunk; the result is laid out so that beta_j of
  // rhs r sits at result[(r * kmax + j) * 2]: stride between lanes is 2 CH
  // within one rhs, 2 kmax between rhs.
  RedArgs r2 = ra;
  r2.result = ra.result + (size_t)rhs * kmax * 2 + (size_t)chunk * 2 * kChunk - (size_t)(rhs * gridDim.y + chunk) * 2 * kChunk;
  r2.stride = 2 * kChunk;
  grid_reduce<2 * kChunk, kVecThreads, R>(red, r2, rhs * gridDim.y + chunk);
}

int launch_multidot(int prec, size_t n, int nrhs, int k, int kmax, const void* W, size_t jstride, const void* w,
                    RedArgs red, cudaStream_t st, const double* pre, const double* post, int cstride) {
  if (k <= 0) return 0;
  if (kmax % kChunk) return -1;
  dim3 grid(red_blocks(n), (k + kChunk - 1) / kChunk, nrhs);
  switch (prec) {
    case 0:
      multidot_kernel<double2><<<grid, kVecThreads, 0, st>>>(n, k, kmax, (const double2*)W, jstride, (const double2*)w,
                                                             red, pre, post, cstride);
      break;
    case 1:
      multidot_kernel<float2><<<grid, kVecThreads, 0, st>>>(n, k, kmax, (const float2*)W, jstride, (const float2*)w,
                                                            red, pre, post, cstride);
      break;
    default: return -1;
  }
  return launched() ? 0 : -1;
}

template <typename S>
__global__ void __launch_bounds__(kVecThreads)
    multiaxpy_kernel(size_t n, int k, int kmax, const double* beta, const S* W, const S* Zb, size_t jstride, S* w,
                     S* z, const S* r, RedArgs ra) {
  typedef typename Store<S>::R R;
  __shared__ cx<R> sb[64];
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n;
  const double* bt = beta + (size_t)rhs * kmax * 2;
  for (int j = threadIdx.x; j < k; j += kVecThreads) sb[j] = mk<R>((R)bt[2 * j], (R)bt[2 * j + 1]);
  __syncthreads();
  R acc[3] = {(R)0, (R)0, (R)0};
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecThreads) {
    cx<R> wv = ldc<R>(w + off, i), zv = ldc<R>(z + off, i);
    // four basis vectors per round: eight independent loads in flight
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      cx<R> a0 = ldc<R>(W + (size_t)(j + 0) * jstride + off, i), c0 = ldc<R>(Zb + (size_t)(j + 0) * jstride + off, i);
      cx<R> a1 = ldc<R>(W + (size_t)(j + 1) * jstride + off, i), c1 = ldc<R>(Zb + (size_t)(j + 1) * jstride + off, i);
      cx<R> a2 = ldc<R>(W + (size_t)(j + 2) * jstride + off, i), c2 = ldc<R>(Zb + (size_t)(j + 2) * jstride + off, i);
      cx<R> a3 = ldc<R>(W + (size_t)(j + 3) * jstride + off, i), c3 = ldc<R>(Zb + (size_t)(j + 3) * jstride + off, i);
      wv = wv - sb[j] * a0;
      zv = zv - sb[j] * c0;
      wv = wv - sb[j + 1] * a1;
      zv = zv - sb[j + 1] * c1;
      wv = wv - sb[j + 2] * a2;
      zv = zv - sb[j + 2] * c2;
      wv = wv - sb[j + 3] * a3;
      zv = zv - sb[j + 3] * c3;
    }
    for (; j < k; ++j) {
      wv = wv - sb[j] * ldc<R>(W + (size_t)j * jstride + off, i);
      zv = zv - sb[j] * ldc<R>(Zb + (size_t)j * jstride + off, i);
    }
    stc(w + off, i, wv);
    stc(z + off, i, zv);
    const cx<R> ws = as_stored<S>(wv);
    const cx<R> d = cmul_conj(ws, ldc<R>(r + off, i));
    acc[0] += d.re;
    acc[1] += d.im;
    acc[2] += norm2(ws);
  }
  if (ra.result) grid_reduce<3, kVecThreads, R>(acc, ra, rhs);
}

int launch_multiaxpy(int prec, size_t n, int nrhs, int k, int kmax, const double* beta, const void* W,
                     const void* Zb, size_t jstride, void* w, void* z, const void* r, RedArgs red2, cudaStream_t st) {
  dim3 grid(vec_blocks(n), nrhs);
  switch (prec) {
    case 0:
      multiaxpy_kernel<double2><<<grid, kVecThreads, 0, st>>>(n, k, kmax, beta, (const double2*)W, (const double2*)Zb,
                                                              jstride, (double2*)w, (double2*)z, (const double2*)r, red2);
      break;
    case 1:
      multiaxpy_kernel<float2><<<grid, kVecThreads, 0, st>>>(n, k, kmax, beta, (const float2*)W, (const float2*)Zb,
                                                             jstride, (float2*)w, (float2*)z, (const float2*)r, red2);
      break;
    default: return -1;
  }
  return launched() ? 0 : -1;
}

template <typename S, typename SX>
__global__ void __launch_bounds__(kVecThreads)
    gcr_update_kernel(size_t n, const double* dots, int dstride, S* w, S* z, SX* x, S* r, RedArgs ra) {
  typedef typename Store<S>::R R;
  typedef typename Store<SX>::R RX;
  const int rhs = blockIdx.y;
  __shared__ double sc[3];
  if (threadIdx.x == 0) {
    const double* d = dots + (size_t)rhs * dstride;
    const double nw2 = d[2];
    double inv = 0.0, ar = 0.0, ai = 0.0;
    if (nw2 > 0.0 && isfinite(nw2)) {
      inv = 1.0 / sqrt(nw2);
      ar = d[0] * inv;
      ai = d[1] * inv;
    }
    sc[0] = inv;
    sc[1] = ar;
    sc[2] = ai;
  }
  __syncthreads();
  const double inv = sc[0], ar = sc[1], ai = sc[2];
  const R s = (R)inv;
  const cx<R> a = mk<R>((R)ar, (R)ai);
  const cx<RX> ax = mk<RX>((RX)ar, (RX)ai);
  const size_t off = (size_t)rhs * n;
  R acc = (R)0;
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecThreads) {
    const cx<R> wv = as_stored<S>(s * ldc<R>(w + off, i));
    const cx<R> zv = as_stored<S>(s * ldc<R>(z + off, i));
    stc(w + off, i, wv);
    stc(z + off, i, zv);
    cx<RX> xv = ldc<RX>(x + off, i);
    xv = cfma(ax, mk<RX>((RX)zv.re, (RX)zv.im), xv);
    stc(x + off, i, xv);
    cx<R> rv = ldc<R>(r + off, i) - a * wv;
    stc(r + off, i, rv);
    acc += norm2(as_stored<S>(rv));
  }
  R red[1] = {acc};
  grid_reduce<1, kVecThreads, R>(red, ra, rhs);
}

int launch_gcr_update(int prec, int xprec, size_t n, int nrhs, const double* dots, int dstride, void* w, void* z,
                      void* x, void* r, RedArgs red, cudaStream_t st) {
  dim3 grid(vec_blocks(n), nrhs);
  if (prec == 0 && xprec == 0)
    gcr_update_kernel<double2, double2><<<grid, kVecThreads, 0, st>>>(n, dots, dstride, (double2*)w, (double2*)z,
                                                                       (double2*)x, (double2*)r, red);
  else if (prec == 1 && xprec == 1)
    gcr_update_kernel<float2, float2><<<grid, kVecThreads, 0, st>>>(n, dots, dstride, (float2*)w, (float2*)z,
                                                                     (float2*)x, (float2*)r, red);
  else if (prec == 1 && xprec == 0)
    gcr_update_kernel<float2, double2><<<grid, kVecThreads, 0, st>>>(n, dots, dstride, (float2*)w, (float2*)z,
                                                                      (double2*)x, (float2*)r, red);
  else
    return -1;
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ GCR with a deferred solution update
// The outer flexible GCR keeps the preconditioned vectors z_j as they come
// out of the cycle and orthonormalises only w = A z against the previous
// w's: A Z = W H with H upper triangular (the Gram-Schmidt coefficients above
// the diagonal, the norms on it).  The residual update r -= alpha_k w_k needs
// only W; at the end of a cycle x += Z y with H y = alpha.  One Gram-Schmidt
// pass (plus a second one on demand) then reads each basis vector once per
// iteration instead of W and Z twice.

// w -= sum_j beta_j W_j, fused <w|r> and ||w||^2 (3 values per right-hand
// side); the coefficients are added to column hk of H.
template <typename S>
__global__ void __launch_bounds__(kVecThreads)
    gs_update_kernel(size_t n, int k, int kmax, const double* beta, const S* W, size_t jstride, S* w, const S* r,
                     RedArgs ra, double2* H, int hk, const double* pre, const double* post, int cstride) {
  typedef typename Store<S>::R R;
  __shared__ cx<R> sb[64];
  const int rhs = blockIdx.y;
  if (gs_pass_skipped(pre, post, cstride, rhs)) return;
  const size_t off = (size_t)rhs * n;
  const double* bt = beta + (size_t)rhs * kmax * 2;
  for (int j = threadIdx.x; j < k; j += kVecThreads) sb[j] = mk<R>((R)bt[2 * j], (R)bt[2 * j + 1]);
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < k; j += kVecThreads) {
      double2& hj = H[((size_t)rhs * kmax + j) * kmax + hk];
      hj.x += bt[2 * j];
      hj.y += bt[2 * j + 1];
    }
  __syncthreads();
  R acc[3] = {(R)0, (R)0, (R)0};
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecThreads) {
    cx<R> wv = ldc<R>(w + off, i);
    int j = 0;
    for (; j + 8 <= k; j += 8) {  // eight independent loads in flight
      cx<R> a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = ldc<R>(W + (size_t)(j + q) * jstride + off, i);
#pragma unroll
      for (int q = 0; q < 8; ++q) wv = wv - sb[j + q] * a[q];
    }
    for (; j < k; ++j) wv = wv - sb[j] * ldc<R>(W + (size_t)j * jstride + off, i);
    stc(w + off, i, wv);
    const cx<R> ws = as_stored<S>(wv);
    const cx<R> d = cmul_conj(ws, ldc<R>(r + off, i));
    acc[0] += d.re;
    acc[1] += d.im;
    acc[2] += norm2(ws);
  }
  grid_reduce<3, kVecThreads, R>(acc, ra, rhs);
}

int launch_gs_update(int prec, size_t n, int nrhs, int k, int kmax, const double* beta, const void* W, size_t jstride,
                     void* w, const void* r, RedArgs red, double2* H, int hk, const double* pre, const double* post,
                     int cstride, cudaStream_t st) {
  if (k <= 0 || k > 64) return k <= 0 ? 0 : -1;
  dim3 grid(vec_blocks(n), nrhs);
  switch (prec) {
    case 0:
      gs_update_kernel<double2><<<grid, kVecThreads, 0, st>>>(n, k, kmax, beta, (const double2*)W, jstride,
                                                              (double2*)w, (const double2*)r, red, H, hk, pre, post,
                                                              cstride);
      break;
    case 1:
      gs_update_kernel<float2><<<grid, kVecThreads, 0, st>>>(n, k, kmax, beta, (const float2*)W, jstride, (float2*)w,
                                                             (const float2*)r, red, H, hk, pre, post, cstride);
      break;
    default: return -1;
  }
  return launched() ? 0 : -1;
}

// w_k = w / ||w||, alpha_k = <w_k|r>, r -= alpha_k w_k, fused ||r||^2; H[k][k]
// = ||w|| and alpha_k are kept for the end of the cycle.  dots = (<w|r>, ||w||^2)
// of the orthogonalised w.
template <typename S>
__global__ void __launch_bounds__(kVecThreads)
    gcr_step_kernel(size_t n, const double* dots, int dstride, S* w, S* r, RedArgs ra, double2* H, double2* alpha,
                    int k, int kmax) {
  typedef typename Store<S>::R R;
  const int rhs = blockIdx.y;
  __shared__ double sc[3];
  if (threadIdx.x == 0) {
    const double* d = dots + (size_t)rhs * dstride;
    const double nw2 = d[2];
    double inv = 0.0, ar = 0.0, ai = 0.0;
    if (nw2 > 0.0 && isfinite(nw2)) {
      inv = 1.0 / sqrt(nw2);
      ar = d[0] * inv;
      ai = d[1] * inv;
    }
    sc[0] = inv;
    sc[1] = ar;
    sc[2] = ai;
    if (blockIdx.x == 0) {
      H[((size_t)rhs * kmax + k) * kmax + k] = make_double2(nw2 > 0.0 ? sqrt(nw2) : 0.0, 0.0);
      alpha[(size_t)rhs * kmax + k] = make_double2(ar, ai);
    }
  }
  __syncthreads();
  const double inv = sc[0], ar = sc[1], ai = sc[2];
  const R s = (R)inv;
  const cx<R> a = mk<R>((R)ar, (R)ai);
  const size_t off = (size_t)rhs * n;
  R acc = (R)0;
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecThreads) {
    const cx<R> wv = as_stored<S>(s * ldc<R>(w + off, i));
    stc(w + off, i, wv);
    const cx<R> rv = ldc<R>(r + off, i) - a * wv;
    stc(r + off, i, rv);
    acc += norm2(as_stored<S>(rv));
  }
  R red[1] = {acc};
  grid_reduce<1, kVecThreads, R>(red, ra, rhs);
}

int launch_gcr_step(int prec, size_t n, int nrhs, const double* dots, int dstride, void* w, void* r, RedArgs red,
                    double2* H, double2* alpha, int k, int kmax, cudaStream_t st) {
  dim3 grid(vec_blocks(n), nrhs);
  if (prec == 0)
    gcr_step_kernel<double2><<<grid, kVecThreads, 0, st>>>(n, dots, dstride, (double2*)w, (double2*)r, red, H, alpha,
                                                           k, kmax);
  else if (prec == 1)
    gcr_step_kernel<float2><<<grid, kVecThreads, 0, st>>>(n, dots, dstride, (float2*)w, (float2*)r, red, H, alpha, k,
                                                          kmax);
  else
    return -1;
  return launched() ? 0 : -1;
}

// y = H^-1 alpha for the k x k upper-triangular H of each right-hand side
// (back substitution in FP64, one thread per right-hand side: k <= 64).
__global__ void back_substitute_kernel(int k, int kmax, const double2* H, const double2* alpha, double2* y) {
  const int rhs = blockIdx.x;
  if (threadIdx.x != 0) return;
  const double2* Hr = H + (size_t)rhs * kmax * kmax;
  const double2* ar = alpha + (size_t)rhs * kmax;
  double2* yr = y + (size_t)rhs * kmax;
  for (int i = k - 1; i >= 0; --i) {
    double sr = ar[i].x, si = ar[i].y;
    for (int j = i + 1; j < k; ++j) {
      const double2 h = Hr[(size_t)i * kmax + j], v = yr[j];
      sr -= h.x * v.x - h.y * v.y;
      si -= h.x * v.y + h.y * v.x;
    }
    const double dd = Hr[(size_t)i * kmax + i].x;
    yr[i] = dd > 0.0 ? make_double2(sr / dd, si / dd) : make_double2(0.0, 0.0);
  }
}

int launch_back_substitute(int nrhs, int k, int kmax, const double2* H, const double2* alpha, double2* y,
                           cudaStream_t st) {
  if (k <= 0) return 0;
  back_substitute_kernel<<<nrhs, 32, 0, st>>>(k, kmax, H, alpha, y);
  return launched() ? 0 : -1;
}

// x += sum_j y_j Z_j (Z in the Krylov precision, x FP64 or the same).
template <typename SZ, typename SX>
__global__ void __launch_bounds__(kVecThreads)
    zcombine_kernel(size_t n, int k, int kmax, const double2* y, const SZ* Z, size_t jstride, SX* x) {
  typedef typename Store<SX>::R RX;
  __shared__ cx<RX> sy[64];
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n;
  for (int j = threadIdx.x; j < k; j += kVecThreads) {
    const double2 v = y[(size_t)rhs * kmax + j];
    sy[j] = mk<RX>((RX)v.x, (RX)v.y);
  }
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecThreads) {
    cx<RX> xv = ldc<RX>(x + off, i);
    int j = 0;
    for (; j + 8 <= k; j += 8) {
      cx<RX> a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = ldc<RX>(Z + (size_t)(j + q) * jstride + off, i);
#pragma unroll
      for (int q = 0; q < 8; ++q) xv = cfma(sy[j + q], a[q], xv);
    }
    for (; j < k; ++j) xv = cfma(sy[j], ldc<RX>(Z + (size_t)j * jstride + off, i), xv);
    stc(x + off, i, xv);
  }
}

int launch_zcombine(int zprec, int xprec, size_t n, int nrhs, int k, int kmax, const double2* y, const void* Z,
                    size_t jstride, void* x, cudaStream_t st) {
  if (k <= 0) return 0;
  if (k > 64) return -1;
  dim3 grid(vec_blocks(n), nrhs);
  if (zprec == 0 && xprec == 0)
    zcombine_kernel<double2, double2><<<grid, kVecThreads, 0, st>>>(n, k, kmax, y, (const double2*)Z, jstride,
                                                                    (double2*)x);
  else if (zprec == 1 && xprec == 0)
    zcombine_kernel<float2, double2><<<grid, kVecThreads, 0, st>>>(n, k, kmax, y, (const float2*)Z, jstride,
                                                                   (double2*)x);
  else
    return -1;
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ Krylov baselines
// out = c0 x0 + c1 x1 + c2 x2 (complex host coefficients, FP64; unused terms
// have a null x; out may be one of the x), with <w|out> and ||out||^2
// reduced when w is given (lane 0, 3 values).
__global__ void __launch_bounds__(kVecThreads) lincomb_kernel(size_t n, LinComb L, RedArgs ra) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecThreads) {
    cx<double> v = zero<double>();
#pragma unroll
    for (int t = 0; t < 3; ++t)
      if (L.x[t]) v = cfma(mk<double>(L.c[t].x, L.c[t].y), ldc<double>(L.x[t], i), v);
    stc(L.out, i, v);
    if (L.w) {
      const cx<double> d = cmul_conj(ldc<double>(L.w, i), v);
      acc[0] += d.re;
      acc[1] += d.im;
      acc[2] += norm2(v);
    }
  }
  if (L.w) grid_reduce<3, kVecThreads, double>(acc, ra, 0);
}

int launch_lincomb(size_t n, const LinComb& L, RedArgs red, cudaStream_t st) {
  lincomb_kernel<<<red_blocks(n), kVecThreads, 0, st>>>(n, L, red);
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ conversions
template <typename SI, typename SO>
__global__ void __launch_bounds__(kVecThreads) convert_kernel(size_t n, const SI* in, SO* out, double s0,
                                                              const double* slot, int sstride, double sexp, int acc) {
  const int rhs = blockIdx.y;
  __shared__ double ss;
  if (threadIdx.x == 0) {
    double s = s0;
    if (slot) {
      const double v = slot[(size_t)rhs * sstride];
      s *= (sexp == 0.5) ? sqrt(v) : (sexp == -0.5 ? (v > 0.0 ? 1.0 / sqrt(v) : 0.0) : pow(v, sexp));
    }
    ss = s;
  }
  __syncthreads();
  const double s = ss;
  const size_t off = (size_t)rhs * n;
  for (size_t i = (size_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecThreads) {
    if (sizeof(typename Store<SI>::R) == 8 || sizeof(typename Store<SO>::R) == 8) {
      cx<double> v = ldc<double>(in + off, i);
      v = s * v;
      if (acc) v = v + ldc<double>(out + off, i);
      stc(out + off, i, v);
    } else {
      cx<float> v = ldc<float>(in + off, i);
      v = (float)s * v;
      if (acc) v = v + ldc<float>(out + off, i);
      stc(out + off, i, v);
    }
  }
}

template <typename SI>
static int convert_to(int pout, dim3 grid, size_t n, const void* in, void* out, double s0, const double* slot,
                      int sstride, double sexp, int acc, cudaStream_t st) {
  const SI* i = (const SI*)in;
  switch (pout) {
    case 0: convert_kernel<SI, double2><<<grid, kVecThreads, 0, st>>>(n, i, (double2*)out, s0, slot, sstride, sexp, acc); break;
    case 1: convert_kernel<SI, float2><<<grid, kVecThreads, 0, st>>>(n, i, (float2*)out, s0, slot, sstride, sexp, acc); break;
    case 2: convert_kernel<SI, __half2><<<grid, kVecThreads, 0, st>>>(n, i, (__half2*)out, s0, slot, sstride, sexp, acc); break;
    case 3:
      convert_kernel<SI, __nv_bfloat162>
          <<<grid, kVecThreads, 0, st>>>(n, i, (__nv_bfloat162*)out, s0, slot, sstride, sexp, acc);
      break;
    default: return -1;
  }
  return launched() ? 0 : -1;
}

int launch_convert(int pin, int pout, size_t n, int nrhs, const void* in, void* out, double s0, const double* slot,
                   int sstride, double sexp, int accumulate, cudaStream_t st) {
  dim3 grid(vec_blocks(n), nrhs);
  switch (pin) {
    case 0: return convert_to<double2>(pout, grid, n, in, out, s0, slot, sstride, sexp, accumulate, st);
    case 1: return convert_to<float2>(pout, grid, n, in, out, s0, slot, sstride, sexp, accumulate, st);
    case 2: return convert_to<__half2>(pout, grid, n, in, out, s0, slot, sstride, sexp, accumulate, st);
    case 3: return convert_to<__nv_bfloat162>(pout, grid, n, in, out, s0, slot, sstride, sexp, accumulate, st);
  }
  return -1;
}

// ------------------------------------------------------------------ layouts
// External [nrhs][V][ncomp] FP64 <-> internal [nrhs] x (field of chunk q).
template <typename S>
__global__ void ext_to_int_kernel(int ncomp, int q, int V, int nrhs, const double2* ext, S* out) {
  const size_t tot = (size_t)nrhs * ncomp * V;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    // i indexes the external layout [r][s][c]
    const int c = (int)(i % ncomp);
    const size_t rs = i / ncomp;
    const int s = (int)(rs % V);
    const size_t r = rs / V;
    const double2 v = ext[i];
    stc(out, r * ncomp * V + fidx_q(c, s, V, q), mk<double>(v.x, v.y));
  }
}

template <typename S>
__global__ void int_to_ext_kernel(int ncomp, int q, int V, int nrhs, const S* in, double2* ext) {
  const size_t tot = (size_t)nrhs * ncomp * V;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    // i indexes the external layout [r][s][c]
    const int c = (int)(i % ncomp);
    const size_t rs = i / ncomp;
    const int s = (int)(rs % V);
    const size_t r = rs / V;
    const cx<double> v = ldc<double>(in, r * ncomp * V + fidx_q(c, s, V, q));
    ext[i] = make_double2(v.re, v.im);
  }
}

static unsigned grid_for(size_t tot) {
  size_t b = (tot + 255) / 256;
  if (b > 8192) b = 8192;
  return (unsigned)(b < 1 ? 1 : b);
}

int launch_ext_to_int(int prec, int ncomp, int q, int V, int nrhs, const void* ext, void* internal, cudaStream_t st) {
  const unsigned g = grid_for((size_t)nrhs * ncomp * V);
  const double2* e = (const double2*)ext;
  switch (prec) {
    case 0: ext_to_int_kernel<double2><<<g, 256, 0, st>>>(ncomp, q, V, nrhs, e, (double2*)internal); break;
    case 1: ext_to_int_kernel<float2><<<g, 256, 0, st>>>(ncomp, q, V, nrhs, e, (float2*)internal); break;
    case 2: ext_to_int_kernel<__half2><<<g, 256, 0, st>>>(ncomp, q, V, nrhs, e, (__half2*)internal); break;
    case 3: ext_to_int_kernel<__nv_bfloat162><<<g, 256, 0, st>>>(ncomp, q, V, nrhs, e, (__nv_bfloat162*)internal); break;
    default: return -1;
  }
  return launched() ? 0 : -1;
}

int launch_int_to_ext(int prec, int ncomp, int q, int V, int nrhs, const void* internal, void* ext, cudaStream_t st) {
  const unsigned g = grid_for((size_t)nrhs * ncomp * V);
  double2* e = (double2*)ext;
  switch (prec) {
    case 0: int_to_ext_kernel<double2><<<g, 256, 0, st>>>(ncomp, q, V, nrhs, (const double2*)internal, e); break;
    case 1: int_to_ext_kernel<float2><<<g, 256, 0, st>>>(ncomp, q, V, nrhs, (const float2*)internal, e); break;
    case 2: int_to_ext_kernel<__half2><<<g, 256, 0, st>>>(ncomp, q, V, nrhs, (const __half2*)internal, e); break;
    case 3:
      int_to_ext_kernel<__nv_bfloat162><<<g, 256, 0, st>>>(ncomp, q, V, nrhs, (const __nv_bfloat162*)internal, e);
      break;
    default: return -1;
  }
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ gamma5
// out = gamma5 in on FP64 level-0 fields of V sites (chunked layout, nrhs of
// them): gamma5 = diag(1, 1, -1, -1) on spin in the chiral basis (Sec. 1), so
// components c = 6..11 change sign.  in and out may be the same.
__global__ void gamma5_kernel(size_t V, size_t tot, const double2* in, double2* out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    const size_t e = i % (12 * V);
    const int c = (int)(e / (4 * V)) * 4 + (int)(e & 3);
    const double2 v = in[i];
    out[i] = c >= 6 ? make_double2(-v.x, -v.y) : v;
  }
}

int launch_gamma5(size_t V, int nrhs, const void* in, void* out, cudaStream_t st) {
  const size_t tot = (size_t)nrhs * 12 * V;
  size_t b = (tot + 255) / 256;
  if (b > 8192) b = 8192;
  gamma5_kernel<<<(unsigned)(b < 1 ? 1 : b), 256, 0, st>>>(V, tot, (const double2*)in, (double2*)out);
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ start vectors
__device__ __forceinline__ uint64_t splitmix64_out(uint64_t state, uint64_t m) {
  uint64_t z = state + (m + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gaussian_starts_kernel(uint64_t seed, int nv, int ncomp, int q, int V, double2* out) {
  const size_t tot = (size_t)nv * ncomp * V;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    // e is the stream index k V ncomp + s ncomp + c of element (k, s, c)
    const int c = (int)(e % ncomp);
    const size_t ks = e / ncomp;
    const int s = (int)(ks % V);
    const size_t k = ks / V;
    const uint64_t x1 = splitmix64_out(seed, 2 * e), x2 = splitmix64_out(seed, 2 * e + 1);
    const double u1 = ((double)(x1 >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = ((double)(x2 >> 11) + 1.0) * 0x1.0p-53;
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[k * ncomp * V + fidx_q(c, s, V, q)] = make_double2(rad * cs, rad * sn);
  }
}

int launch_gaussian_starts(uint64_t seed, int nv, int ncomp, int q, int V, void* out, cudaStream_t st) {
  gaussian_starts_kernel<<<grid_for((size_t)nv * ncomp * V), 256, 0, st>>>(seed, nv, ncomp, q, V, (double2*)out);
  return launched() ? 0 : -1;
}

}  // namespace wmg
