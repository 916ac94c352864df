// Restriction R = P^+ and prolongation P (Sec. 3, Eq. 3.2 and the text
// after it) for many right-hand sides on tensor cores.
//
// Per aggregate B and chirality chi both are dense complex products with the
// aggregate's block of P, P_B (nv x len, len = ncomp/2 * |B| components):
//   restriction   out (nv x R)  = conj(P_B) (nv x len) * v (len x R)
//   prolongation  out (len x R) = P_B^T (len x nv) * x_c (nv x R)
// The kernels on CUDA cores read P_B once per right-hand side; here one CTA
// per (B, chi) reads it once for all R (R <= 64), which is what bounds the
// multi-right-hand-side transfer: at nv = 24 and 16-bit storage P is 1152 B
// per fine site, as much as 24 right-hand sides of the vectors themselves.
//
// Arithmetic: mma.sync m16n8k16 with 16-bit inputs (FP16 or BF16, the
// storage type of the fine vectors and of P) and FP32 accumulation, in the
// real embedding of the complex product: with P = Pr + i Pi,
//   conj(P) v : re = Pr vr + Pi vi,  im = Pr vi - Pi vr
//   P x       : re = Pr xr - Pi xi,  im = Pr xi + Pi xr
// so each 16 x 16 fragment pair of P feeds four MMAs (-Pi is Pi with the
// sign bits flipped).  Operands are staged in shared memory as separate real
// and imaginary planes, K contiguous, so every fragment register is one
// 32-bit shared load.  Summation order is fixed (K ascending per warp slice,
// slices added in order), so results are deterministic.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"

namespace wmg {

static inline bool launched() { return launch_ok(); }

template <typename T>
struct MmaT;
template <>
struct MmaT<__half> {
  typedef __half2 T2;
  static __device__ __forceinline__ __half from(float x) { return __float2half_rn(x); }
  static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
};
template <>
struct MmaT<__nv_bfloat16> {
  typedef __nv_bfloat162 T2;
  static __device__ __forceinline__ __nv_bfloat16 from(float x) { return __float2bfloat16_rn(x); }
  static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
};

__device__ __forceinline__ uint32_t ld32(const void* p) { return *(const uint32_t*)p; }

// A stored complex value as its two 16-bit planes: a bit move when the
// storage type is the MMA type, a rounding when it is FP32.
template <typename T>
__device__ __forceinline__ void planes(const typename MmaT<T>::T2 v, T& re, T& im) {
  re = v.x;
  im = v.y;
}
template <typename T>
__device__ __forceinline__ void planes(const float2 v, T& re, T& im) {
  re = MmaT<T>::from(v.x);
  im = MmaT<T>::from(v.y);
}
__device__ __forceinline__ uint32_t neg2(uint32_t v) { return v ^ 0x80008000u; }

// Fine site of aggregate B, aggregate-local site s (x fastest in both).
__device__ __forceinline__ int agg_site_t(const Agg& g, int B, int s) {
  int cb[4], cl[4], cf[4];
  site_coords(B, g.Lc, cb);
  site_coords(s, g.blk, cl);
#pragma unroll
  for (int m = 0; m < 4; ++m) cf[m] = cb[m] * g.blk[m] + cl[m];
  return site_index(cf, g.L);
}

constexpr int kTThreads = 256;  // 8 warps
constexpr int kTK = 128;        // K (restriction) or M (prolongation) chunk staged per step
constexpr int kTKs = kTK + 8;   // row stride of a staged plane: rows gid = 0..7 of a fragment fall in distinct banks

// ------------------------------------------------------------------ restriction
// CTA (B, chi).  Warp w owns M tile mt = w % MT (rows k of P) and the K steps
// ks = w / MT, w / MT + 8 / MT, ... of every chunk; the 8 / MT slices are
// added through shared memory at the end.
template <typename T, typename SI, typename SO, int NT8>
__global__ void __launch_bounds__(kTThreads)
    restrict_mma_kernel(const Agg g, const typename MmaT<T>::T2* P, const SI* in, SO* out, int R, int sidx_off) {
  typedef typename MmaT<T>::T2 T2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int MT = (g.nv + 15) / 16, Mp = MT * 16, NS = 8 / MT;
  const int Rp = NT8 * 8;
  T* Ps = (T*)smem_raw;          // [2][Mp][kTKs]
  T* Vs = Ps + 2 * Mp * kTKs;    // [2][Rp][kTKs]
  int* sidx = (int*)(smem_raw + sidx_off);  // fine site of each aggregate-local site
  const int B = blockIdx.x, chi = blockIdx.y;
  const int r0 = blockIdx.z * Rp;  // first right-hand side of this CTA (launch-shape split)
  const int len = g.nhalf * g.bsites;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int mt = warp % MT, ks0 = warp / MT;
  const T2* Pb = P + ((size_t)B * 2 + chi) * g.nv * len;
  for (int s = threadIdx.x; s < g.bsites; s += kTThreads) sidx[s] = agg_site_t(g, B, s);
  float accr[NT8][4], acci[NT8][4];
#pragma unroll
  for (int q = 0; q < NT8; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) accr[q][e] = acci[q][e] = 0.f;
  for (int e0 = 0; e0 < len; e0 += kTK) {
    __syncthreads();
    // staging: thread t owns column el = t % kTK of the chunk and the rows
    // t / kTK, t / kTK + 2, ... (the aggregate site of el is looked up once)
    {
      const int el = threadIdx.x % kTK, rr = threadIdx.x / kTK, e = e0 + el;
      const bool live = e < len;
      const T zero16 = MmaT<T>::from(0.f);
#pragma unroll 4
      for (int k = rr; k < Mp; k += kTThreads / kTK) {
        T re = zero16, im = zero16;
        if (live && k < g.nv) planes<T>(Pb[(size_t)k * len + e], re, im);
        Ps[(size_t)k * kTKs + el] = re;
        Ps[(size_t)(Mp + k) * kTKs + el] = im;
      }
      size_t base = 0;
      if (live) {
        const int c = e / g.bsites, s = e - c * g.bsites;
        base = fidx_q(chi * g.nhalf + c, sidx[s], g.V, g.q);
      }
      const size_t rstride = (size_t)g.ncomp * g.V;
#pragma unroll 4
      for (int r = rr; r < Rp; r += kTThreads / kTK) {
        T re = zero16, im = zero16;
        if (live && r0 + r < R) planes<T>(in[(size_t)(r0 + r) * rstride + base], re, im);
        Vs[(size_t)r * kTKs + el] = re;
        Vs[(size_t)(Rp + r) * kTKs + el] = im;
      }
    }
    __syncthreads();
    for (int ks = ks0; ks < kTK / 16; ks += NS) {
      const int kc = ks * 16 + 2 * tig;
      const T* pr0 = Ps + (size_t)(mt * 16 + gid) * kTKs + kc;
      const T* pi0 = Ps + (size_t)(Mp + mt * 16 + gid) * kTKs + kc;
      const uint32_t Ar[4] = {ld32(pr0), ld32(pr0 + 8 * kTKs), ld32(pr0 + 8), ld32(pr0 + 8 * kTKs + 8)};
      const uint32_t Ai[4] = {ld32(pi0), ld32(pi0 + 8 * kTKs), ld32(pi0 + 8), ld32(pi0 + 8 * kTKs + 8)};
      const uint32_t An[4] = {neg2(Ai[0]), neg2(Ai[1]), neg2(Ai[2]), neg2(Ai[3])};
#pragma unroll
      for (int q = 0; q < NT8; ++q) {
        const T* vr = Vs + (size_t)(q * 8 + gid) * kTKs + kc;
        const T* vi = Vs + (size_t)(Rp + q * 8 + gid) * kTKs + kc;
        const uint32_t br0 = ld32(vr), br1 = ld32(vr + 8), bi0 = ld32(vi), bi1 = ld32(vi + 8);
        MmaT<T>::mma(accr[q], Ar, br0, br1);  // Pr vr
        MmaT<T>::mma(accr[q], Ai, bi0, bi1);  // + Pi vi
        MmaT<T>::mma(acci[q], Ar, bi0, bi1);  // Pr vi
        MmaT<T>::mma(acci[q], An, br0, br1);  // - Pi vr
      }
    }
  }
  // add the K slices: slice ks0 > 0 parks its tile, slice 0 sums in slice order
  __syncthreads();
  float* red = (float*)smem_raw;  // [8 warps][NT8][2][4][32]
  if (ks0 > 0) {
#pragma unroll
    for (int q = 0; q < NT8; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        red[((((size_t)warp * NT8 + q) * 2 + 0) * 4 + e) * 32 + lane] = accr[q][e];
        red[((((size_t)warp * NT8 + q) * 2 + 1) * 4 + e) * 32 + lane] = acci[q][e];
      }
  }
  __syncthreads();
  if (ks0 != 0) return;
  for (int sl = 1; sl < NS; ++sl) {
    const int w2 = sl * MT + mt;
#pragma unroll
    for (int q = 0; q < NT8; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        accr[q][e] += red[((((size_t)w2 * NT8 + q) * 2 + 0) * 4 + e) * 32 + lane];
        acci[q][e] += red[((((size_t)w2 * NT8 + q) * 2 + 1) * 4 + e) * 32 + lane];
      }
  }
#pragma unroll
  for (int q = 0; q < NT8; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = mt * 16 + gid + (e >= 2 ? 8 : 0);
      const int r = r0 + q * 8 + 2 * tig + (e & 1);
      if (k < g.nv && r < R)
        stc(out, ((size_t)r * 2 * g.nv + chi * g.nv + k) * g.Vc + B, mk<float>(accr[q][e], acci[q][e]));
    }
}

// ------------------------------------------------------------------ prolongation
// CTA (B, chi); chunks of kTK rows e of P_B^T, warp w the 16 rows w * 16.. of
// the chunk, all of K = nv (padded to KT * 16) and all right-hand sides.
template <typename T, typename SI, typename SO, int NT8>
__global__ void __launch_bounds__(kTThreads)
    prolong_mma_kernel(const Agg g, const typename MmaT<T>::T2* P, const SI* in, SO* out, int R, int sidx_off) {
  typedef typename MmaT<T>::T2 T2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int KT = (g.nv + 15) / 16, Kp = KT * 16, Kps = Kp + 8;  // Kps: bank-spread row stride
  const int Rp = NT8 * 8;
  T* Xs = (T*)smem_raw;          // [2][Rp][Kps]
  T* Pt = Xs + 2 * Rp * Kps;     // [2][kTK][Kps]
  int* sidx = (int*)(smem_raw + sidx_off);
  const int B = blockIdx.x, chi = blockIdx.y;
  const int r0 = blockIdx.z * Rp;  // first right-hand side of this CTA (launch-shape split)
  const int len = g.nhalf * g.bsites;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const T2* Pb = P + ((size_t)B * 2 + chi) * g.nv * len;
  for (int s = threadIdx.x; s < g.bsites; s += kTThreads) sidx[s] = agg_site_t(g, B, s);
  for (int t = threadIdx.x; t < Rp * Kp; t += kTThreads) {
    const int r = t / Kp, k = t % Kp;
    T re = MmaT<T>::from(0.f), im = re;
    if (r0 + r < R && k < g.nv) planes<T>(in[((size_t)(r0 + r) * 2 * g.nv + chi * g.nv + k) * g.Vc + B], re, im);
    Xs[(size_t)r * Kps + k] = re;
    Xs[(size_t)(Rp + r) * Kps + k] = im;
  }
  for (int e0 = 0; e0 < len; e0 += kTK) {
    __syncthreads();
    {
      const int el = threadIdx.x % kTK, rr = threadIdx.x / kTK, e = e0 + el;
      const T zero16 = MmaT<T>::from(0.f);
#pragma unroll 4
      for (int k = rr; k < Kp; k += kTThreads / kTK) {
        T re = zero16, im = zero16;
        if (e < len && k < g.nv) planes<T>(Pb[(size_t)k * len + e], re, im);
        Pt[(size_t)el * Kps + k] = re;
        Pt[(size_t)(kTK + el) * Kps + k] = im;
      }
    }
    __syncthreads();
    float accr[NT8][4], acci[NT8][4];
#pragma unroll
    for (int q = 0; q < NT8; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) accr[q][e] = acci[q][e] = 0.f;
    for (int ks = 0; ks < KT; ++ks) {
      const int kc = ks * 16 + 2 * tig;
      const T* pr0 = Pt + (size_t)(warp * 16 + gid) * Kps + kc;
      const T* pi0 = Pt + (size_t)(kTK + warp * 16 + gid) * Kps + kc;
      const uint32_t Ar[4] = {ld32(pr0), ld32(pr0 + 8 * Kps), ld32(pr0 + 8), ld32(pr0 + 8 * Kps + 8)};
      const uint32_t Ai[4] = {ld32(pi0), ld32(pi0 + 8 * Kps), ld32(pi0 + 8), ld32(pi0 + 8 * Kps + 8)};
      const uint32_t An[4] = {neg2(Ai[0]), neg2(Ai[1]), neg2(Ai[2]), neg2(Ai[3])};
#pragma unroll
      for (int q = 0; q < NT8; ++q) {
        const T* xr = Xs + (size_t)(q * 8 + gid) * Kps + kc;
        const T* xi = Xs + (size_t)(Rp + q * 8 + gid) * Kps + kc;
        const uint32_t br0 = ld32(xr), br1 = ld32(xr + 8), bi0 = ld32(xi), bi1 = ld32(xi + 8);
        MmaT<T>::mma(accr[q], Ar, br0, br1);  // Pr xr
        MmaT<T>::mma(accr[q], An, bi0, bi1);  // - Pi xi
        MmaT<T>::mma(acci[q], Ar, bi0, bi1);  // Pr xi
        MmaT<T>::mma(acci[q], Ai, br0, br1);  // + Pi xr
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = e0 + warp * 16 + gid + 8 * h;
      if (e >= len) continue;
      const int c = e / g.bsites, s = e - c * g.bsites;
      const size_t o = fidx_q(chi * g.nhalf + c, sidx[s], g.V, g.q);
#pragma unroll
      for (int q = 0; q < NT8; ++q)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int r = r0 + q * 8 + 2 * tig + j;
          if (r < R) stc(out, (size_t)r * g.ncomp * g.V + o, mk<float>(accr[q][2 * h + j], acci[q][2 * h + j]));
        }
    }
  }
}

// ------------------------------------------------------------------ launchers
// Dynamic shared memory: the staged operands (or, in the restriction, the
// K-slice partial sums that reuse them), then the aggregate's site table at
// the returned offset.
static size_t restrict_smem(const Agg& g, int NT8, size_t* sidx_off) {
  const int MT = (g.nv + 15) / 16;
  const size_t stage = (size_t)2 * (MT * 16 + NT8 * 8) * kTKs * 2;
  const size_t red = (size_t)8 * NT8 * 2 * 4 * 32 * 4;
  *sidx_off = ((stage > red ? stage : red) + 15) / 16 * 16;
  return *sidx_off + (size_t)g.bsites * 4;
}

static size_t prolong_smem(const Agg& g, int NT8, size_t* sidx_off) {
  const int Kps = (g.nv + 15) / 16 * 16 + 8;
  *sidx_off = ((size_t)2 * (NT8 * 8 + kTK) * Kps * 2 + 15) / 16 * 16;
  return *sidx_off + (size_t)g.bsites * 4;
}

bool transfer_mma_ok(const Agg& g, int nrhs) {
  const int MT = (g.nv + 15) / 16;
  return nrhs >= 2 && nrhs <= 64 && (MT == 1 || MT == 2 || MT == 4) && g.ncomp % 2 == 0 && g.bsites <= 8192;
}

// Launch shapes: variant v puts kXTiles[v] tiles of 8 right-hand sides in a CTA
// (the admissible ones for nrhs, in this order); the default holds them all.
static const int kXTiles[] = {8, 4, 2, 1, 3, 6};
constexpr int kXVariants = 6;

int transfer_mma_variants(int nrhs) {
  const int NT8 = (nrhs + 7) / 8;
  int nv = 0;
  for (int v = 0; v < kXVariants; ++v) nv += kXTiles[v] <= NT8 ? 1 : 0;
  return nv;
}

static int tiles_of(int nrhs, int variant) {
  const int all = (nrhs + 7) / 8;
  if (variant < 0) return all;
  int seen = -1;
  for (int v = 0; v < kXVariants; ++v)
    if (kXTiles[v] <= all && ++seen == variant) return kXTiles[v];
  return all;
}

template <typename T, typename SI, typename SO>
static int restrict_mma_t(const Agg& g, const void* P, const void* in, void* out, int nrhs, cudaStream_t st,
                          int variant) {
  const int NT8 = tiles_of(nrhs, variant);
  size_t so = 0;
  const size_t sm = restrict_smem(g, NT8, &so);
  const dim3 grid(g.Vc, 2, ((nrhs + 7) / 8 + NT8 - 1) / NT8);
#define WMG_RM(K)                                                                                              \
  {                                                                                                            \
    auto kern = restrict_mma_kernel<T, SI, SO, K>;                                                             \
    if (sm > 48 * 1024) allow_big_smem(kern);                                                                  \
    kern<<<grid, kTThreads, sm, st>>>(g, (const typename MmaT<T>::T2*)P, (const SI*)in, (SO*)out, nrhs, (int)so); \
  }
  switch (NT8) {
    case 1: WMG_RM(1); break;
    case 2: WMG_RM(2); break;
    case 3: WMG_RM(3); break;
    case 4: WMG_RM(4); break;
    case 5: WMG_RM(5); break;
    case 6: WMG_RM(6); break;
    case 7: WMG_RM(7); break;
    case 8: WMG_RM(8); break;
    default: return -1;
  }
#undef WMG_RM
  return launched() ? 0 : -1;
}

template <typename T, typename SI, typename SO>
static int prolong_mma_t(const Agg& g, const void* P, const void* in, void* out, int nrhs, cudaStream_t st,
                         int variant) {
  const int NT8 = tiles_of(nrhs, variant);
  size_t so = 0;
  const size_t sm = prolong_smem(g, NT8, &so);
  const dim3 grid(g.Vc, 2, ((nrhs + 7) / 8 + NT8 - 1) / NT8);
#define WMG_PM(K)                                                                                              \
  {                                                                                                            \
    auto kern = prolong_mma_kernel<T, SI, SO, K>;                                                              \
    if (sm > 48 * 1024) allow_big_smem(kern);                                                                  \
    kern<<<grid, kTThreads, sm, st>>>(g, (const typename MmaT<T>::T2*)P, (const SI*)in, (SO*)out, nrhs, (int)so); \
  }
  switch (NT8) {
    case 1: WMG_PM(1); break;
    case 2: WMG_PM(2); break;
    case 3: WMG_PM(3); break;
    case 4: WMG_PM(4); break;
    case 5: WMG_PM(5); break;
    case 6: WMG_PM(6); break;
    case 7: WMG_PM(7); break;
    case 8: WMG_PM(8); break;
    default: return -1;
  }
#undef WMG_PM
  return launched() ? 0 : -1;
}

// (vector-in, P, vector-out) precision triples with 16-bit P: 2 = FP16, 3 = BF16, 1 = FP32.
int launch_restrict_mma(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                        cudaStream_t st, int variant) {
  if (pin == 2 && pP == 2 && pout == 1)
    return restrict_mma_t<__half, __half2, float2>(g, P, in, out, nrhs, st, variant);
  if (pin == 3 && pP == 3 && pout == 1)
    return restrict_mma_t<__nv_bfloat16, __nv_bfloat162, float2>(g, P, in, out, nrhs, st, variant);
  if (pin == 2 && pP == 2 && pout == 2)
    return restrict_mma_t<__half, __half2, __half2>(g, P, in, out, nrhs, st, variant);
  if (pin == 3 && pP == 3 && pout == 3)
    return restrict_mma_t<__nv_bfloat16, __nv_bfloat162, __nv_bfloat162>(g, P, in, out, nrhs, st, variant);
  return -1;
}

int launch_prolong_mma(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                       cudaStream_t st, int variant) {
  if (pin == 1 && pP == 2 && pout == 2)
    return prolong_mma_t<__half, float2, __half2>(g, P, in, out, nrhs, st, variant);
  if (pin == 1 && pP == 3 && pout == 3)
    return prolong_mma_t<__nv_bfloat16, float2, __nv_bfloat162>(g, P, in, out, nrhs, st, variant);
  if (pin == 2 && pP == 2 && pout == 2)
    return prolong_mma_t<__half, __half2, __half2>(g, P, in, out, nrhs, st, variant);
  if (pin == 3 && pP == 3 && pout == 3)
    return prolong_mma_t<__nv_bfloat16, __nv_bfloat162, __nv_bfloat162>(g, P, in, out, nrhs, st, variant);
  return -1;
}

}  // namespace wmg
