// Shared device helpers: complex arithmetic, storage precisions, deterministic reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace wmg {

// Launch checks: a launcher reads (and so clears) the thread's last CUDA error
// right after its launch; the error is kept here so that the caller's message
// names it.
inline thread_local cudaError_t tl_launch_error = cudaSuccess;
inline bool launch_ok() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) tl_launch_error = e;
  return e == cudaSuccess;
}
inline cudaError_t take_launch_error() {
  const cudaError_t e = tl_launch_error;
  tl_launch_error = cudaSuccess;
  return e;
}

// Dynamic shared memory above 48 KB needs a per-kernel opt-in.  The attribute
// is global to the kernel, so a value chosen per launch would race between
// host threads launching the same kernel with different sizes; every caller
// sets the device's maximum instead, the same value from any thread (the
// amount a launch really uses still sets its occupancy).
inline int smem_optin_bytes() {
  static const int v = [] {
    int d = 0, x = 48 * 1024;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, d) !=
                                                 cudaSuccess) {
      cudaGetLastError();
      x = 48 * 1024;
    }
    return x;
  }();
  return v;
}
// Streaming multiprocessors of the current device (queried once; 152 on GB300).
inline int sm_count() {
  static const int v = [] {
    int d = 0, x = 152;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&x, cudaDevAttrMultiProcessorCount, d) != cudaSuccess ||
        x < 1) {
      cudaGetLastError();
      x = 152;
    }
    return x;
  }();
  return v;
}

template <typename K>
inline void allow_big_smem(K kern) {
  cudaFuncAttributes fa;
  int bytes = smem_optin_bytes();
  if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess)
    bytes -= (int)fa.sharedSizeBytes;  // the opt-in limit covers static plus dynamic shared memory
  else
    cudaGetLastError();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
    cudaGetLastError();
}


// ------------------------------------------------------------------ complex
template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> zero() {
  return mk<R>(R(0), R(0));
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) {
  return mk<R>(a.re + b.re, a.im + b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) {
  return mk<R>(a.re - b.re, a.im - b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) {
  return mk<R>(s * a.re, s * a.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> conj(cx<R> a) {
  return mk<R>(a.re, -a.im);
}
// conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ cx<R> cmul_conj(cx<R> a, cx<R> b) {
  return mk<R>(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// acc + a * b
template <typename R>
__host__ __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ cx<R> cfma_conj(cx<R> a, cx<R> b, cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> times_i(cx<R> a) {
  return mk<R>(-a.im, a.re);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> times_minus_i(cx<R> a) {
  return mk<R>(a.im, -a.re);
}
template <typename R>
__host__ __device__ __forceinline__ R norm2(cx<R> a) {
  return a.re * a.re + a.im * a.im;
}

// ------------------------------------------------------------------ storage
// A complex element stored as two reals of type T; arithmetic type R.
template <typename T>
struct Store;

template <>
struct Store<double2> {
  typedef double R;
  static __device__ __forceinline__ cx<double> ld(const double2* p, size_t i) {
    double2 v = p[i];
    return mk<double>(v.x, v.y);
  }
  static __device__ __forceinline__ void st(double2* p, size_t i, cx<double> v) {
    p[i] = make_double2(v.re, v.im);
  }
};
template <>
struct Store<float2> {
  typedef float R;
  static __device__ __forceinline__ cx<float> ld(const float2* p, size_t i) {
    float2 v = p[i];
    return mk<float>(v.x, v.y);
  }
  static __device__ __forceinline__ void st(float2* p, size_t i, cx<float> v) {
    p[i] = make_float2(v.re, v.im);
  }
};
template <>
struct Store<__half2> {
  typedef float R;
  static __device__ __forceinline__ cx<float> ld(const __half2* p, size_t i) {
    float2 v = __half22float2(p[i]);
    return mk<float>(v.x, v.y);
  }
  static __device__ __forceinline__ void st(__half2* p, size_t i, cx<float> v) {
    p[i] = __floats2half2_rn(v.re, v.im);
  }
};
template <>
struct Store<__nv_bfloat162> {
  typedef float R;
  static __device__ __forceinline__ cx<float> ld(const __nv_bfloat162* p, size_t i) {
    float2 v = __bfloat1622float2(p[i]);
    return mk<float>(v.x, v.y);
  }
  static __device__ __forceinline__ void st(__nv_bfloat162* p, size_t i, cx<float> v) {
    p[i] = __floats2bfloat162_rn(v.re, v.im);
  }
};

// The value a complex number has after a round trip through storage T.
template <typename T>
__device__ __forceinline__ cx<typename Store<T>::R> as_stored(cx<typename Store<T>::R> v);
template <>
__device__ __forceinline__ cx<double> as_stored<double2>(cx<double> v) { return v; }
template <>
__device__ __forceinline__ cx<float> as_stored<float2>(cx<float> v) { return v; }
template <>
__device__ __forceinline__ cx<float> as_stored<__half2>(cx<float> v) {
  float2 f = __half22float2(__floats2half2_rn(v.re, v.im));
  return mk<float>(f.x, f.y);
}
template <>
__device__ __forceinline__ cx<float> as_stored<__nv_bfloat162>(cx<float> v) {
  float2 f = __bfloat1622float2(__floats2bfloat162_rn(v.re, v.im));
  return mk<float>(f.x, f.y);
}

// Read a complex value of any storage into arithmetic type R2.
template <typename R2, typename T>
__device__ __forceinline__ cx<R2> ldc(const T* p, size_t i) {
  cx<typename Store<T>::R> v = Store<T>::ld(p, i);
  return mk<R2>((R2)v.re, (R2)v.im);
}
template <typename T, typename R2>
__device__ __forceinline__ void stc(T* p, size_t i, cx<R2> v) {
  typedef typename Store<T>::R R;
  Store<T>::st(p, i, mk<R>((R)v.re, (R)v.im));
}

// Bytes of one stored complex element per precision code (0 f64, 1 f32, 2 f16, 3 bf16).
__host__ __device__ inline size_t cx_bytes(int prec) { return prec == 0 ? 16 : (prec == 1 ? 8 : 4); }

// ------------------------------------------------------------------ lattice geometry
// Sites are lexicographic with x fastest; directions d = 0 (self),
// 1 + 2 mu (n + mu), 2 + 2 mu (n - mu); periodic boundaries.
__host__ __device__ __forceinline__ void site_coords(int s, const int (&L)[4], int (&c)[4]) {
  c[0] = s % L[0];
  s /= L[0];
  c[1] = s % L[1];
  s /= L[1];
  c[2] = s % L[2];
  c[3] = s / L[2];
}
__host__ __device__ __forceinline__ int site_index(const int (&c)[4], const int (&L)[4]) {
  return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]));
}
__host__ __device__ __forceinline__ int neighbor(const int (&c)[4], const int (&L)[4], int d) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  if (d > 0) {
    const int mu = (d - 1) >> 1;
    if (d & 1)
      n[mu] = (n[mu] + 1 == L[mu]) ? 0 : n[mu] + 1;
    else
      n[mu] = (n[mu] == 0) ? L[mu] - 1 : n[mu] - 1;
  }
  return site_index(n, L);
}

// ------------------------------------------------------------------ field layouts
// Level-0 fields (12 complex components c = spin * 3 + colour per site) are
// stored in three chunks of four components, each chunk site-major:
// component c of site s at complex index ((c / 4) V + s) 4 + c % 4 (per
// right-hand side; wilson_hop.cuh gives the reason).  Coarse-level fields
// are component-major, [ncomp][V].  The chunk q of a field is 4 or 1.
__host__ __device__ __forceinline__ size_t fidx(int c, size_t s, size_t V) {
  return (((size_t)(c >> 2) * V + s) << 2) + (c & 3);
}
__host__ __device__ __forceinline__ size_t fidx_q(int c, size_t s, size_t V, int q) {
  return q == 4 ? fidx(c, s, V) : (size_t)c * V + s;
}

// ------------------------------------------------------------------ reductions
// Deterministic grid reductions: every block writes NV partial doubles, then
// the last block to finish (atomic ticket after a fence) sums the partials of
// all blocks in block order and writes the result.  Summation order is fixed
// by the launch shape, never by scheduling.  Each reduction "lane" (one per
// right-hand side) owns a ticket counter that the last block resets to 0.
struct RedArgs {
  double* partials;   // [nlanes][gridDim.x][NV]
  unsigned* tickets;  // [nlanes]
  double* result;     // [nlanes][stride]
  int stride;         // doubles between lanes in result
};

template <int NV, int NT, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* smem /* NV * NT/32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) smem[k * (NT / 32) + warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T s = lane < NT / 32 ? smem[k * (NT / 32) + lane] : (T)0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[k] = s;  // valid in thread 0
    }
  }
  __syncthreads();
}

// Finish a grid reduction for lane `ln` whose blocks are blockIdx.x in
// [0, gridDim.x).  Call from every thread of every block with the thread's
// partial values of type T; NT = blockDim.x (a multiple of 32, <= 1024).
// The tree inside a block runs in T (FP32 for the FP32 / 16-bit kernels:
// FP64 arithmetic is scarce on this part); the sum over blocks runs in FP64.
template <int NV, int NT, typename T>
__device__ __forceinline__ void grid_reduce(T (&v)[NV], const RedArgs& ra, int ln) {
  __shared__ T smem_t[NV * (NT / 32)];
  __shared__ double smem_d[NV * (NT / 32)];
  __shared__ bool last;
  block_sum<NV, NT, T>(v, smem_t);
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
    double* dst = ra.partials + ((size_t)ln * nb + blockIdx.x) * NV;
#pragma unroll
    for (int k = 0; k < NV; ++k) dst[k] = (double)v[k];
    __threadfence();
    unsigned t = atomicAdd(ra.tickets + ln, 1u);
    last = (t == (unsigned)nb - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double w[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) w[k] = 0.0;
  for (int b = threadIdx.x; b < nb; b += NT) {
    const double* src = ra.partials + ((size_t)ln * nb + b) * NV;
#pragma unroll
    for (int k = 0; k < NV; ++k) w[k] += __ldcg(src + k);
  }
  block_sum<NV, NT, double>(w, smem_d);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) ra.result[(size_t)ln * ra.stride + k] = w[k];
    ra.tickets[ln] = 0u;
  }
}

}  // namespace wmg
