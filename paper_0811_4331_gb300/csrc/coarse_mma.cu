// Coarse 9-point stencil on tensor cores for many right-hand sides.
//
// (A_c y)(B) = sum_d C_d(B) y(B + d)  (A_c = P^+ A P, Sec. 2) is, per coarse
// site B, one dense contraction O (n x R) = [C_0 .. C_8](B) (n x 9n) * Y (9n x R)
// over the R right-hand sides.  In the real embedding
//   [O_re; O_im] = [[C_re, -C_im], [C_im, C_re]] [Y_re; Y_im]
// it runs as BF16 mma.sync m16n8k16 with FP32 accumulation.  One warp owns
// a pair of 16-row tiles (the real rows and the imaginary rows of the same
// 16 components), so each 16x16 block of C_re and C_im is loaded once and
// used by four MMAs (C_re Y_re, -C_im Y_im into the real tile; C_im Y_re,
// C_re Y_im into the imaginary tile; -C_im is C_im with the sign bits
// flipped).  The operator is stored at setup in MMA fragment order,
// [B][d][tile][kstep][re|im][lane][8 x bf16], so a warp reads 512 contiguous
// bytes per fragment; the right-hand sides of the 9 neighbours are staged in
// shared memory as BF16, [d][r][re..., im...].  n is padded to a multiple of
// 16 and R to a multiple of 8 with zeros.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace wmg {

static inline bool launched() { return launch_ok(); }

// ------------------------------------------------------------------ operator in fragment order
// One thread per (B, d, tile, kstep, part, lane): 8 bf16 of the A fragment
// of m16n8k16 (rows gid, gid + 8; columns 2 tig, 2 tig + 1, and + 8).
__global__ void mma_pack_kernel(const double2* C, int n, int npad, int V, uint4* out) {
  const int T = npad / 16;  // row tiles = k steps per half
  const size_t per_site = (size_t)9 * T * T * 2 * 32;
  const size_t tot = per_site * V;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    size_t q = e;
    const int lane = (int)(q % 32);
    q /= 32;
    const int part = (int)(q % 2);
    q /= 2;
    const int s = (int)(q % T);
    q /= T;
    const int t = (int)(q % T);
    q /= T;
    const int d = (int)(q % 9);
    const int B = (int)(q / 9);
    const int gid = lane >> 2, tig = lane & 3;
    const int rows[2] = {t * 16 + gid, t * 16 + gid + 8};
    const int cols[4] = {s * 16 + 2 * tig, s * 16 + 2 * tig + 1, s * 16 + 2 * tig + 8, s * 16 + 2 * tig + 9};
    // a0 a1: (r0, c0 c1); a2 a3: (r1, c0 c1); a4 a5: (r0, c2 c3); a6 a7: (r1, c2 c3)
    const int ri[8] = {0, 0, 1, 1, 0, 0, 1, 1};
    const int ci[8] = {0, 1, 0, 1, 2, 3, 2, 3};
    __nv_bfloat16 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = rows[ri[k]], j = cols[ci[k]];
      double x = 0.0;
      if (i < n && j < n) {
        const double2 c = C[((size_t)(d * n + i) * n + j) * V + B];
        x = part ? c.y : c.x;
      }
      v[k] = __float2bfloat16_rn((float)x);
    }
    uint4 w;
    w.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
    w.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
    w.z = (uint32_t)__bfloat16_as_ushort(v[4]) | ((uint32_t)__bfloat16_as_ushort(v[5]) << 16);
    w.w = (uint32_t)__bfloat16_as_ushort(v[6]) | ((uint32_t)__bfloat16_as_ushort(v[7]) << 16);
    out[e] = w;
  }
}

size_t mma_pack_bytes(int n, int V) {
  const int npad = (n + 15) / 16 * 16, T = npad / 16;
  return (size_t)9 * T * T * 2 * 32 * 16 * V;
}

int launch_mma_pack(const double2* C, int n, int V, void* out, cudaStream_t st) {
  const int npad = (n + 15) / 16 * 16, T = npad / 16;
  const size_t tot = (size_t)9 * T * T * 2 * 32 * V;
  size_t b = (tot + 255) / 256;
  if (b > 8192) b = 8192;
  mma_pack_kernel<<<(unsigned)b, 256, 0, st>>>(C, n, npad, V, (uint4*)out);
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ apply
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <typename S, int NT8>
__global__ void coarse_mma_kernel(const uint4* Cf, const S* in, S* out, const S* y2, int L0, int L1, int L2, int L3,
                                  int n, int npad, int R, float a, float c, const double* shift) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* Ys = (__nv_bfloat16*)smem_raw;  // [9][Rpad][2 npad]
  const int L[4] = {L0, L1, L2, L3};
  const int V = L0 * L1 * L2 * L3;
  const int B = blockIdx.x;
  const int r0 = blockIdx.y * NT8 * 8;  // first right-hand side of this CTA (launch-shape split)
  const int Rpad = NT8 * 8;
  const int T = npad / 16;
  const int KW = 2 * npad;  // one neighbour's row of Ys: re then im
  int cB[4];
  site_coords(B, L, cB);
  // stage the 9 neighbours' right-hand sides as BF16
  for (int e = threadIdx.x; e < 9 * Rpad * npad; e += blockDim.x) {
    const int j = e % npad, r = (e / npad) % Rpad, d = e / (npad * Rpad);
    float re = 0.f, im = 0.f;
    if (j < n && r0 + r < R) {
      const cx<float> v = ldc<float>(in, ((size_t)(r0 + r) * n + j) * V + neighbor(cB, L, d));
      re = v.re;
      im = v.im;
    }
    Ys[((size_t)d * Rpad + r) * KW + j] = __float2bfloat16_rn(re);
    Ys[((size_t)d * Rpad + r) * KW + npad + j] = __float2bfloat16_rn(im);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = warp;  // row-tile pair owned by this warp
  if (t >= T) return;
  const int gid = lane >> 2, tig = lane & 3;
  float accr[NT8][4], acci[NT8][4];
#pragma unroll
  for (int q = 0; q < NT8; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k) accr[q][k] = acci[q][k] = 0.f;
  const uint4* Cs = Cf + (size_t)B * 9 * T * T * 2 * 32;
  // (d, s) steps in order; the operator fragments of the next two steps are
  // loaded while the current one runs, so three 512-byte loads per warp stay
  // in flight (the stencil is bound by the latency of these reads otherwise)
  const int KS = 9 * T;
  auto frag = [&](int k) { return ((((size_t)(k / T) * T + t) * T + (k % T)) * 2) * 32 + lane; };
  uint4 f0r = __ldg(Cs + frag(0)), f0i = __ldg(Cs + frag(0) + 32);
  uint4 f1r = f0r, f1i = f0i;
  if (KS > 1) {
    f1r = __ldg(Cs + frag(1));
    f1i = __ldg(Cs + frag(1) + 32);
  }
  for (int k = 0; k < KS; ++k) {
    const int d = k / T, s = k - d * T;
    const __nv_bfloat16* Yd = Ys + (size_t)d * Rpad * KW;
    const uint4 fr = f0r, fi = f0i;
    f0r = f1r;
    f0i = f1i;
    if (k + 2 < KS) {
      f1r = __ldg(Cs + frag(k + 2));
      f1i = __ldg(Cs + frag(k + 2) + 32);
    }
    {
      const uint32_t Ar[4] = {fr.x, fr.y, fr.z, fr.w};
      const uint32_t Ai[4] = {fi.x, fi.y, fi.z, fi.w};
      const uint32_t An[4] = {fi.x ^ 0x80008000u, fi.y ^ 0x80008000u, fi.z ^ 0x80008000u, fi.w ^ 0x80008000u};
#pragma unroll
      for (int q = 0; q < NT8; ++q) {
        const __nv_bfloat16* col = Yd + (size_t)(q * 8 + gid) * KW;
        const int k0 = s * 16 + 2 * tig;
        const uint32_t yr0 = *(const uint32_t*)(col + k0), yr1 = *(const uint32_t*)(col + k0 + 8);
        const uint32_t yi0 = *(const uint32_t*)(col + npad + k0), yi1 = *(const uint32_t*)(col + npad + k0 + 8);
        mma_bf16(accr[q], Ar, yr0, yr1);  // C_re Y_re
        mma_bf16(accr[q], An, yi0, yi1);  // -C_im Y_im
        mma_bf16(acci[q], Ai, yr0, yr1);  // C_im Y_re
        mma_bf16(acci[q], Ar, yi0, yi1);  // C_re Y_im
      }
    }
  }
  // epilogue: rows t*16 + gid (+8), right-hand sides q*8 + 2 tig (+1)
#pragma unroll
  for (int q = 0; q < NT8; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = t * 16 + gid + (k >= 2 ? 8 : 0);
      const int r = r0 + q * 8 + 2 * tig + (k & 1);
      if (i < n && r < R) {
        const size_t o = ((size_t)r * n + i) * V + B;
        cx<float> acc = mk<float>(accr[q][k], acci[q][k]);
        if (shift) acc = cfma(mk<float>((float)shift[r], 0.f), ldc<float>(in, o), acc);
        cx<float> v = mk<float>(a * acc.re, a * acc.im);
        if (y2) v = v + c * ldc<float>(y2, o);
        stc(out, o, v);
      }
    }
}

// Launch shapes: variant v splits the right-hand sides over CTAs in groups of
// kMmaTiles[v] tiles of 8 (each output's arithmetic is the same in every shape).
static const int kMmaTiles[] = {8, 4, 2, 1, 3, 6};
constexpr int kMmaVariants = 6;

int coarse_mma_variants(int R) {
  const int NT8 = (R + 7) / 8;
  int nv = 0;
  for (int v = 0; v < kMmaVariants; ++v) nv += kMmaTiles[v] <= NT8 ? 1 : 0;
  return nv;
}

int launch_coarse_mma(int prec, const void* Cf, const void* in, void* out, const void* y2, const int L[4], int n, int R,
                      double a, double c, cudaStream_t st, int variant, const double* shift) {
  if (prec != 1 && prec != 3) return -1;
  const int npad = (n + 15) / 16 * 16, T = npad / 16;
  const int V = L[0] * L[1] * L[2] * L[3];
  const int NT8all = (R + 7) / 8;
  int NT8 = NT8all;  // default: one CTA per coarse site holds every right-hand side
  if (variant >= 0) {
    int seen = -1;
    for (int v = 0; v < kMmaVariants; ++v)
      if (kMmaTiles[v] <= NT8all && ++seen == variant) NT8 = kMmaTiles[v];
  }
  const int splits = (NT8all + NT8 - 1) / NT8;
  const size_t sm = (size_t)9 * NT8 * 8 * 2 * npad * sizeof(__nv_bfloat16);
  if (sm > 200 * 1024 || T > 32) return -1;
#define WMG_MMA(S, K)                                                                                    \
  {                                                                                                      \
    auto kern = coarse_mma_kernel<S, K>;                                                                 \
    if (sm > 48 * 1024) allow_big_smem(kern);                                                            \
    kern<<<dim3(V, splits), 32 * T, sm, st>>>((const uint4*)Cf, (const S*)in, (S*)out, (const S*)y2, L[0], L[1],    \
                                              L[2], L[3], n,                                                       \
                                npad, R, (float)a, (float)c, shift);                                     \
  }
#define WMG_MMA_R(S)                       \
  switch (NT8) {                           \
    case 1: WMG_MMA(S, 1); break;          \
    case 2: WMG_MMA(S, 2); break;          \
    case 3: WMG_MMA(S, 3); break;          \
    case 4: WMG_MMA(S, 4); break;          \
    case 5: WMG_MMA(S, 5); break;          \
    case 6: WMG_MMA(S, 6); break;          \
    case 7: WMG_MMA(S, 7); break;          \
    case 8: WMG_MMA(S, 8); break;          \
    default: return -1;                    \
  }
  if (prec == 1) {
    WMG_MMA_R(float2)
  } else {
    WMG_MMA_R(__nv_bfloat162)
  }
#undef WMG_MMA_R
#undef WMG_MMA
  return launched() ? 0 : -1;
}

}  // namespace wmg
