// Per-site pieces of the Wilson hopping term shared by the stencil kernel
// and the Galerkin coarse-operator build: link loads with 12-real
// reconstruction, SU(3) multiplies, and one projected hop in the chiral
// gamma basis g_k = [[0, -i s_k], [i s_k, 0]], g_t = [[0, 1], [1, 0]]
// (Sec. 1 operator).  With psi = (u, d) (upper / lower spin pairs) and
// g_mu = [[0, X], [X^-1, 0]], (1 - g_mu) psi = (h, -X^-1 h) with
// h = u - X d, and (1 + g_mu) psi = (h', X^-1 h') with h' = u + X d.
#pragma once
#include "common.cuh"

namespace wmg {

template <typename R>
struct Link {
  cx<R> m[3][3];
};

template <typename R, typename G, int NL>
__device__ __forceinline__ void load_link(Link<R>& u, const G* U, int mu, int V, int site) {
#pragma unroll
  for (int k = 0; k < NL; ++k) u.m[k / 3][k % 3] = ldc<R>(U, (size_t)(mu * NL + k) * V + site);
  if (NL == 6) {
    // third row of an SU(3) matrix: conj(row0 x row1)
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

// Input of a hop: component i (= comp * V + site) of the field, as a value of
// arithmetic type R.  StoredIn reads a stored field; the MR-fused stencil
// passes one that forms r - c p on the fly.
template <typename R, typename S>
struct StoredIn {
  const S* p;
  __device__ __forceinline__ cx<R> operator()(size_t i) const { return ldc<R>(p, i); }
};

// One hop: project psi(nbr) with (1 - g_mu) (FWD) or (1 + g_mu), multiply by
// U or U^+, reconstruct the lower spin pair, accumulate into acc.
template <int MU, bool FWD, typename R, typename In>
__device__ __forceinline__ void hop_from(cx<R> (&acc)[4][3], const In& in, int V, int nbr, const Link<R>& u) {
  cx<R> h0[3], h1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<R> u0 = in((size_t)(0 * 3 + a) * V + nbr);
    cx<R> u1 = in((size_t)(1 * 3 + a) * V + nbr);
    cx<R> d0 = in((size_t)(2 * 3 + a) * V + nbr);
    cx<R> d1 = in((size_t)(3 * 3 + a) * V + nbr);
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

template <int MU, bool FWD, typename R, typename S>
__device__ __forceinline__ void hop(cx<R> (&acc)[4][3], const S* in, int V, int nbr, const Link<R>& u) {
  hop_from<MU, FWD, R>(acc, StoredIn<R, S>{in}, V, nbr, u);
}

}  // namespace wmg
