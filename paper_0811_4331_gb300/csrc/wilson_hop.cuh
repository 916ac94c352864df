// Level-0 data layouts and the per-site pieces of the Wilson hopping term
// (Sec. 1 operator), shared by the stencil kernels, the even-odd kernels and
// the Galerkin build: vectorised spinor and link loads, 12-real SU(3)
// reconstruction, and one projected hop in the chiral gamma basis
// g_k = [[0, -i s_k], [i s_k, 0]], g_t = [[0, 1], [1, 0]].  With psi = (u, d)
// (upper / lower spin pairs) and g_mu = [[0, X], [X^-1, 0]],
// (1 - g_mu) psi = (h, -X^-1 h) with h = u - X d, and (1 + g_mu) psi =
// (h', X^-1 h') with h' = u + X d.
//
// Level-0 fields (12 complex components c = spin * 3 + colour per site) are
// stored in three chunks of four components, each chunk site-major: component
// c of site s sits at complex index ((c / 4) V + s) 4 + c % 4 (per right-hand
// side).  One chunk of one site is 16 bytes in FP16/BF16, 32 in FP32 and 64
// in FP64, so a neighbour's spinor arrives in 3, 6 or 12 sixteen-byte loads
// and every such load of a warp covers consecutive 16-byte slots.
//
// Links (two stored rows, the third rebuilt, except FP64 which keeps all
// nine elements k = row * 3 + col), link mu of site s, stored element k:
//   FP16 / BF16 (4-byte complex): k < 4 at (mu V + s) 4 + k, k = 4, 5 at
//     16 V + (mu V + s) 2 + k - 4   (one 16-byte and one 8-byte load);
//   FP32 (8-byte complex): ((3 mu + k / 2) V + s) 2 + k % 2  (three 16-byte loads);
//   FP64 (16-byte complex): (9 mu + k) V + s.
#pragma once
#include "common.cuh"

namespace wmg {

// Complex index of stored element k of link (mu, s), storage element type G.
// (The link arrays hold 4 NL V < 2^32 complex elements: offsets in 32 bits.)
template <typename G, int NL>
__host__ __device__ __forceinline__ size_t lidx(int mu, int k, size_t s, size_t V) {
  const unsigned u = (unsigned)s, W = (unsigned)V;
  if constexpr (sizeof(G) == 4)
    return k < 4 ? (size_t)((((unsigned)mu * W + u) << 2) + k) : (size_t)(16u * W + (((unsigned)mu * W + u) << 1) + (k - 4));
  else if constexpr (sizeof(G) == 8)
    return (size_t)((((unsigned)(3 * mu + (k >> 1)) * W + u) << 1) + (k & 1));
  else
    return (size_t)(((unsigned)(mu * NL + k)) * W + u);
}

// ------------------------------------------------------------------ conversions of 4-byte complex words
template <typename S>
__device__ __forceinline__ cx<float> w2c(unsigned w);
template <>
__device__ __forceinline__ cx<float> w2c<__half2>(unsigned w) {
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w));
  return mk<float>(f.x, f.y);
}
// BF16 -> FP32 is exact bit placement (byte permutes on the integer pipe).
template <>
__device__ __forceinline__ cx<float> w2c<__nv_bfloat162>(unsigned w) {
  return mk<float>(__uint_as_float(__byte_perm(w, 0u, 0x1044u)), __uint_as_float(__byte_perm(w, 0u, 0x3244u)));
}
template <typename S>
__device__ __forceinline__ unsigned c2w(cx<float> v);
template <>
__device__ __forceinline__ unsigned c2w<__half2>(cx<float> v) {
  const __half2 h = __floats2half2_rn(v.re, v.im);
  return *reinterpret_cast<const unsigned*>(&h);
}
template <>
__device__ __forceinline__ unsigned c2w<__nv_bfloat162>(cx<float> v) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.re, v.im);
  return *reinterpret_cast<const unsigned*>(&h);
}

// ------------------------------------------------------------------ chunk loads / stores
// Four consecutive complex elements starting at complex index i (a multiple of 4), as type R.
template <typename R, typename S>
__device__ __forceinline__ void ld_chunk(const S* p, size_t i, cx<R> (&v)[4]) {
  if constexpr (sizeof(S) == 4) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(p + i));
    const cx<float> a = w2c<S>(q.x), b = w2c<S>(q.y), c = w2c<S>(q.z), d = w2c<S>(q.w);
    v[0] = mk<R>((R)a.re, (R)a.im);
    v[1] = mk<R>((R)b.re, (R)b.im);
    v[2] = mk<R>((R)c.re, (R)c.im);
    v[3] = mk<R>((R)d.re, (R)d.im);
  } else if constexpr (sizeof(S) == 8) {
    const float4 q0 = __ldg(reinterpret_cast<const float4*>(p + i));
    const float4 q1 = __ldg(reinterpret_cast<const float4*>(p + i) + 1);
    v[0] = mk<R>((R)q0.x, (R)q0.y);
    v[1] = mk<R>((R)q0.z, (R)q0.w);
    v[2] = mk<R>((R)q1.x, (R)q1.y);
    v[3] = mk<R>((R)q1.z, (R)q1.w);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 q = __ldg(reinterpret_cast<const double2*>(p + i) + k);
      v[k] = mk<R>((R)q.x, (R)q.y);
    }
  }
}
// The same through the L2 only (for data written earlier in the same launch).
template <typename R, typename S>
__device__ __forceinline__ void ld_chunk_cg(const S* p, size_t i, cx<R> (&v)[4]) {
  if constexpr (sizeof(S) == 4) {
    const uint4 q = __ldcg(reinterpret_cast<const uint4*>(p + i));
    const cx<float> a = w2c<S>(q.x), b = w2c<S>(q.y), c = w2c<S>(q.z), d = w2c<S>(q.w);
    v[0] = mk<R>((R)a.re, (R)a.im);
    v[1] = mk<R>((R)b.re, (R)b.im);
    v[2] = mk<R>((R)c.re, (R)c.im);
    v[3] = mk<R>((R)d.re, (R)d.im);
  } else if constexpr (sizeof(S) == 8) {
    const float4 q0 = __ldcg(reinterpret_cast<const float4*>(p + i));
    const float4 q1 = __ldcg(reinterpret_cast<const float4*>(p + i) + 1);
    v[0] = mk<R>((R)q0.x, (R)q0.y);
    v[1] = mk<R>((R)q0.z, (R)q0.w);
    v[2] = mk<R>((R)q1.x, (R)q1.y);
    v[3] = mk<R>((R)q1.z, (R)q1.w);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 q = __ldcg(reinterpret_cast<const double2*>(p + i) + k);
      v[k] = mk<R>((R)q.x, (R)q.y);
    }
  }
}
template <typename S, typename R>
__device__ __forceinline__ void st_chunk(S* p, size_t i, const cx<R> (&v)[4]) {
  if constexpr (sizeof(S) == 4) {
    uint4 q;
    q.x = c2w<S>(mk<float>((float)v[0].re, (float)v[0].im));
    q.y = c2w<S>(mk<float>((float)v[1].re, (float)v[1].im));
    q.z = c2w<S>(mk<float>((float)v[2].re, (float)v[2].im));
    q.w = c2w<S>(mk<float>((float)v[3].re, (float)v[3].im));
    *reinterpret_cast<uint4*>(p + i) = q;
  } else if constexpr (sizeof(S) == 8) {
    reinterpret_cast<float4*>(p + i)[0] = make_float4((float)v[0].re, (float)v[0].im, (float)v[1].re, (float)v[1].im);
    reinterpret_cast<float4*>(p + i)[1] = make_float4((float)v[2].re, (float)v[2].im, (float)v[3].re, (float)v[3].im);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) reinterpret_cast<double2*>(p + i)[k] = make_double2((double)v[k].re, (double)v[k].im);
  }
}

// All 12 components of site s of a level-0 field with V sites (offsets within
// one field in 32-bit arithmetic: 12 V < 2^32).
template <typename R, typename S>
__device__ __forceinline__ void ld_spinor(const S* in, size_t V, size_t s, cx<R> (&v)[12]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    cx<R> t[4];
    ld_chunk<R, S>(in, (size_t)(((unsigned)j * (unsigned)V + (unsigned)s) << 2), t);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[4 * j + k] = t[k];
  }
}

// ------------------------------------------------------------------ links
template <typename R>
struct Link {
  cx<R> m[3][3];
};

// Link mu of site `site` (V sites in the layout), third row rebuilt as
// conj(row0 x row1) when only two rows are stored (exact for SU(3)).
template <typename R, typename G, int NL>
__device__ __forceinline__ void load_link(Link<R>& u, const G* U, int mu, int V, int site) {
  if constexpr (sizeof(G) == 4) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(U + lidx<G, NL>(mu, 0, site, V)));
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(U + lidx<G, NL>(mu, 4, site, V)));
    const unsigned w[6] = {q.x, q.y, q.z, q.w, r.x, r.y};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const cx<float> f = w2c<G>(w[k]);
      u.m[k / 3][k % 3] = mk<R>((R)f.re, (R)f.im);
    }
  } else if constexpr (sizeof(G) == 8) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(U + lidx<G, NL>(mu, 2 * j, site, V)));
      u.m[(2 * j) / 3][(2 * j) % 3] = mk<R>((R)q.x, (R)q.y);
      u.m[(2 * j + 1) / 3][(2 * j + 1) % 3] = mk<R>((R)q.z, (R)q.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NL; ++k) u.m[k / 3][k % 3] = ldc<R>(U, lidx<G, NL>(mu, k, site, V));
  }
  if (NL == 6) {
    u.m[2][0] = conj(u.m[0][1] * u.m[1][2] - u.m[0][2] * u.m[1][1]);
    u.m[2][1] = conj(u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2]);
    u.m[2][2] = conj(u.m[0][0] * u.m[1][1] - u.m[0][1] * u.m[1][0]);
  }
}

// g = U h (DAG = false) or U^+ h (DAG = true) for one colour vector.
template <bool DAG, typename R>
__device__ __forceinline__ void su3_mul(const Link<R>& u, const cx<R> (&h)[3], cx<R> (&g)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<R> s = zero<R>();
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) s = DAG ? cfma_conj(u.m[bb][a], h[bb], s) : cfma(u.m[a][bb], h[bb], s);
    g[a] = s;
  }
}

// One hop on a loaded neighbour spinor psi: project with (1 - g_mu) (FWD) or
// (1 + g_mu), multiply by U or U^+, reconstruct the lower spin pair,
// accumulate into acc.
template <int MU, bool FWD, typename R>
__device__ __forceinline__ void hop_vals(cx<R> (&acc)[4][3], const cx<R> (&psi)[12], const Link<R>& u) {
  cx<R> h0[3], h1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cx<R> u0 = psi[a], u1 = psi[3 + a], d0 = psi[6 + a], d1 = psi[9 + a];
    if (MU == 0) {
      h0[a] = FWD ? u0 + times_i(d1) : u0 - times_i(d1);
      h1[a] = FWD ? u1 + times_i(d0) : u1 - times_i(d0);
    } else if (MU == 1) {
      h0[a] = FWD ? u0 + d1 : u0 - d1;
      h1[a] = FWD ? u1 - d0 : u1 + d0;
    } else if (MU == 2) {
      h0[a] = FWD ? u0 + times_i(d0) : u0 - times_i(d0);
      h1[a] = FWD ? u1 - times_i(d1) : u1 + times_i(d1);
    } else {
      h0[a] = FWD ? u0 - d0 : u0 + d0;
      h1[a] = FWD ? u1 - d1 : u1 + d1;
    }
  }
  cx<R> g0[3], g1[3];
  su3_mul<!FWD>(u, h0, g0);
  su3_mul<!FWD>(u, h1, g1);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc[0][a] = acc[0][a] + g0[a];
    acc[1][a] = acc[1][a] + g1[a];
    cx<R> l0, l1;
    if (MU == 0) {
      l0 = FWD ? times_minus_i(g1[a]) : times_i(g1[a]);
      l1 = FWD ? times_minus_i(g0[a]) : times_i(g0[a]);
    } else if (MU == 1) {
      l0 = FWD ? zero<R>() - g1[a] : g1[a];
      l1 = FWD ? g0[a] : zero<R>() - g0[a];
    } else if (MU == 2) {
      l0 = FWD ? times_minus_i(g0[a]) : times_i(g0[a]);
      l1 = FWD ? times_i(g1[a]) : times_minus_i(g1[a]);
    } else {
      l0 = FWD ? zero<R>() - g0[a] : g0[a];
      l1 = FWD ? zero<R>() - g1[a] : g1[a];
    }
    acc[2][a] = acc[2][a] + l0;
    acc[3][a] = acc[3][a] + l1;
  }
}

// One hop from site nbr of a stored level-0 field with V sites.
template <int MU, bool FWD, typename R, typename S>
__device__ __forceinline__ void hop(cx<R> (&acc)[4][3], const S* in, int V, int nbr, const Link<R>& u) {
  cx<R> psi[12];
  ld_spinor<R, S>(in, (size_t)V, (size_t)nbr, psi);
  hop_vals<MU, FWD, R>(acc, psi, u);
}

// ------------------------------------------------------------------ packed FP32 hop
// The same hop in FP32 with paired arithmetic (__ffma2_rn, two FP32 lanes per
// instruction): the two projected spin rows h0, h1 travel as one pair per real
// part, so the SU(3) multiply of both rows costs one paired FMA per real
// product.  Every lane does the scalar operations of hop_vals on its row;
// only the association of the final sums differs.  Accumulators: upper spins
// (0, 1) in up*, lower spins as (2, 3) pairs for z and t hops (ls*) and as
// (3, 2) pairs for x and y hops (lw*), whose lower rows swap spins.
struct Acc2 {
  float2 upr[3], upi[3];
  float2 lsr[3], lsi[3];
  float2 lwr[3], lwi[3];
};

__device__ __forceinline__ void acc2_zero(Acc2& A) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
    A.upr[i] = A.upi[i] = A.lsr[i] = A.lsi[i] = A.lwr[i] = A.lwi[i] = make_float2(0.f, 0.f);
}
// Component c (spin * 3 + colour) of the accumulated hopping term.
__device__ __forceinline__ cx<float> acc2_get(const Acc2& A, int c) {
  const int sp = c / 3, a = c % 3;
  if (sp == 0) return mk<float>(A.upr[a].x, A.upi[a].x);
  if (sp == 1) return mk<float>(A.upr[a].y, A.upi[a].y);
  if (sp == 2) return mk<float>(A.lsr[a].x + A.lwr[a].y, A.lsi[a].x + A.lwi[a].y);
  return mk<float>(A.lsr[a].y + A.lwr[a].x, A.lsi[a].y + A.lwi[a].x);
}

template <int MU, bool FWD>
__device__ __forceinline__ void hop_packed(Acc2& A, const cx<float> (&psi)[12], const Link<float>& u) {
  // projection h = u + s X d per spin row (X = i for x and z hops)
  constexpr bool XI = (MU == 0 || MU == 2);
  constexpr int DA = (MU <= 1) ? 9 : 6, DB = (MU <= 1) ? 6 : 9;
  constexpr float s0 = (MU == 3) ? (FWD ? -1.f : 1.f) : (FWD ? 1.f : -1.f);
  constexpr float s1 = (MU == 0) ? (FWD ? 1.f : -1.f) : (FWD ? -1.f : 1.f);
  float2 hr[3], hi[3], nh[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 ure = make_float2(psi[a].re, psi[3 + a].re), uim = make_float2(psi[a].im, psi[3 + a].im);
    if (XI) {
      hr[a] = __ffma2_rn(make_float2(-s0, -s1), make_float2(psi[DA + a].im, psi[DB + a].im), ure);
      hi[a] = __ffma2_rn(make_float2(s0, s1), make_float2(psi[DA + a].re, psi[DB + a].re), uim);
    } else {
      hr[a] = __ffma2_rn(make_float2(s0, s1), make_float2(psi[DA + a].re, psi[DB + a].re), ure);
      hi[a] = __ffma2_rn(make_float2(s0, s1), make_float2(psi[DA + a].im, psi[DB + a].im), uim);
    }
    nh[a] = FWD ? __fmul2_rn(make_float2(-1.f, -1.f), hi[a]) : __fmul2_rn(make_float2(-1.f, -1.f), hr[a]);
  }
  // g = U h (FWD) or U^+ h
  float2 gr[3], gi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const cx<float> m = FWD ? u.m[a][b] : u.m[b][a];
      const float2 mr = make_float2(m.re, m.re), mi = make_float2(m.im, m.im);
      if (b == 0) {
        gr[a] = __fmul2_rn(mr, hr[0]);
        gi[a] = __fmul2_rn(mr, hi[0]);
      } else {
        gr[a] = __ffma2_rn(mr, hr[b], gr[a]);
        gi[a] = __ffma2_rn(mr, hi[b], gi[a]);
      }
      if (FWD) {
        gr[a] = __ffma2_rn(mi, nh[b], gr[a]);
        gi[a] = __ffma2_rn(mi, hr[b], gi[a]);
      } else {
        gr[a] = __ffma2_rn(mi, hi[b], gr[a]);
        gi[a] = __ffma2_rn(mi, nh[b], gi[a]);
      }
    }
  }
  // accumulate the upper rows, and the lower rows l = t Y g (Y = i for x and z hops)
  constexpr float t0 = (MU == 1) ? (FWD ? 1.f : -1.f) : (FWD ? -1.f : 1.f);
  constexpr float t1 = (MU == 2) ? (FWD ? 1.f : -1.f) : (FWD ? -1.f : 1.f);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    A.upr[a] = __fadd2_rn(A.upr[a], gr[a]);
    A.upi[a] = __fadd2_rn(A.upi[a], gi[a]);
    float2& lr = (MU <= 1) ? A.lwr[a] : A.lsr[a];
    float2& li = (MU <= 1) ? A.lwi[a] : A.lsi[a];
    if (XI) {
      lr = __ffma2_rn(make_float2(-t0, -t1), gi[a], lr);
      li = __ffma2_rn(make_float2(t0, t1), gr[a], li);
    } else {
      lr = __ffma2_rn(make_float2(t0, t1), gr[a], lr);
      li = __ffma2_rn(make_float2(t0, t1), gi[a], li);
    }
  }
}

}  // namespace wmg
