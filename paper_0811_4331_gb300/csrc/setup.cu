// Setup kernels of the adaptive multigrid (FP64 throughout):
//
// * blockwise Gram-Schmidt of the candidate vectors into P (Sec. 2, adaptive
//   step 3 and Eq. 2.3: P V_c = V with P^+ P = 1), one aggregate and
//   chirality per CTA (chirality kept intact, Sec. 3 after Eq. 3.2 and the
//   blocking of Sec. 5), classical Gram-Schmidt applied twice in candidate
//   order;
// * the Galerkin coarse operator A_c = P^+ A P (Sec. 2) as a 9-point stencil:
//   column j of every block C_d'(B) comes from one CTA per aggregate that
//   applies each fine hop A_d to the prolongator column j and projects the
//   result onto the rows of P, sorting each fine hop into the coarse
//   direction d' it crosses (d' = 0 when it stays inside the aggregate).
#include "common.cuh"
#include "kernels.h"
#include "wilson_hop.cuh"

#include <cooperative_groups.h>

namespace wmg {

static inline bool launched() { return launch_ok(); }

__device__ __forceinline__ int agg_site2(const Agg& g, int B, int s) {
  int cb[4], cl[4], cf[4];
  site_coords(B, g.Lc, cb);
  site_coords(s, g.blk, cl);
#pragma unroll
  for (int m = 0; m < 4; ++m) cf[m] = cb[m] * g.blk[m] + cl[m];
  return site_index(cf, g.L);
}

// Deterministic block sum of one complex value (FP64); result valid in all threads.
template <int NT>
__device__ __forceinline__ cx<double> block_csum(cx<double> v, double* sm) {
  double a[2] = {v.re, v.im};
  block_sum<2, NT, double>(a, sm);
  __shared__ double out[2];
  if (threadIdx.x == 0) {
    out[0] = a[0];
    out[1] = a[1];
  }
  __syncthreads();
  cx<double> r = mk<double>(out[0], out[1]);
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------ block Gram-Schmidt
constexpr int kGsMaxNv = 128;  // candidates per level the block Gram-Schmidt takes
constexpr int kGsCluster = 2;  // CTAs (SMs) per aggregate and chirality: FP64 is this part's scarce pipe

// Sum of NV values over the block, then over the CTAs of the cluster in rank
// order (the same total in every CTA and thread).  part: NV doubles of this
// CTA's shared memory, sm: NV * NT / 32 doubles of scratch.
template <int NV, int NT>
__device__ __forceinline__ void cluster_sum(double (&a)[NV], double* sm, double* part) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  block_sum<NV, NT, double>(a, sm);
  if (threadIdx.x == 0)
#pragma unroll
    for (int u = 0; u < NV; ++u) part[u] = a[u];
  cl.sync();  // every CTA's partial is written
#pragma unroll
  for (int u = 0; u < NV; ++u) {
    double t = 0.0;
    for (int r = 0; r < (int)cl.num_blocks(); ++r) t += cl.map_shared_rank(part, r)[u];
    a[u] = t;
  }
  cl.sync();  // every CTA has read every partial before any is overwritten
}

// One classical Gram-Schmidt pass of q (this CTA's elements e in [e0, e1),
// this thread's e0 + tid + m NT) against the k earlier vectors
// p_j = base + j len: all k overlaps first (eight per reduction), then one
// combined update.
template <int NT>
__device__ __forceinline__ void cgs_pass(const double2* base, int k, int len, int e0, int e1, double2* q, double* sm,
                                         double* part, cx<double>* dots) {
  for (int j0 = 0; j0 < k; j0 += 8) {
    double a[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) a[u] = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += NT) {
      const cx<double> qe = mk<double>(q[e].x, q[e].y);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < k) {  // a += conj(p) q: four FP64 FMAs
          const double2 pv = base[(size_t)(j0 + u) * len + e];
          a[2 * u] = fma(pv.x, qe.re, fma(pv.y, qe.im, a[2 * u]));
          a[2 * u + 1] = fma(pv.x, qe.im, fma(-pv.y, qe.re, a[2 * u + 1]));
        }
    }
    cluster_sum<16, NT>(a, sm, part);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if ((int)threadIdx.x == u && j0 + u < k) dots[j0 + u] = mk<double>(a[2 * u], a[2 * u + 1]);
    __syncthreads();
  }
  for (int e = e0 + threadIdx.x; e < e1; e += NT) {
    cx<double> v = mk<double>(q[e].x, q[e].y);
    for (int j = 0; j < k; ++j) {  // v -= d_j p_j, four FP64 FMAs
      const double2 pv = base[(size_t)j * len + e];
      const cx<double> d = dots[j];
      v.re = fma(-d.re, pv.x, fma(d.im, pv.y, v.re));
      v.im = fma(-d.re, pv.y, fma(-d.im, pv.x, v.im));
    }
    q[e] = make_double2(v.re, v.im);
  }
  __syncthreads();
}

// One cluster of kGsCluster CTAs per (aggregate B, chirality chi), each CTA a
// contiguous share of the block's elements: the candidates restricted to the
// block, orthonormalised in candidate order by classical Gram-Schmidt applied
// twice (each pass removes the overlaps with all earlier vectors at once).
template <int NT>
__global__ void __cluster_dims__(kGsCluster, 1, 1) __launch_bounds__(NT)
    block_gs_kernel(const Agg g, const double2* cand, double2* P, int* err) {
  __shared__ double sm[16 * (NT / 32)];
  __shared__ double part[16];
  __shared__ cx<double> dots[kGsMaxNv];
  const int pair = blockIdx.x / kGsCluster, rank = blockIdx.x % kGsCluster;
  const int B = pair >> 1, chi = pair & 1;
  const int nv = g.nv, nh = g.nhalf, bs = g.bsites;
  const int len = nh * bs;
  const int e0 = (int)((long)rank * len / kGsCluster), e1 = (int)((long)(rank + 1) * len / kGsCluster);
  double2* base = P + ((size_t)B * 2 + chi) * nv * len;
  for (int k = 0; k < nv; ++k) {
    double2* q = base + (size_t)k * len;
    // gather candidate k restricted to (B, chi)
    double nrm[1] = {0.0};
    for (int e = e0 + threadIdx.x; e < e1; e += NT) {
      const int c = e / bs, s = e - c * bs;
      const double2 v = cand[(size_t)k * g.ncomp * g.V + fidx_q(chi * nh + c, agg_site2(g, B, s), g.V, g.q)];
      q[e] = v;
      nrm[0] += v.x * v.x + v.y * v.y;
    }
    cluster_sum<1, NT>(nrm, sm, part);
    const double orig = nrm[0];
    if (k > 0) {
      cgs_pass<NT>(base, k, len, e0, e1, q, sm, part, dots);
      cgs_pass<NT>(base, k, len, e0, e1, q, sm, part, dots);
    }
    nrm[0] = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += NT) nrm[0] += q[e].x * q[e].x + q[e].y * q[e].y;
    cluster_sum<1, NT>(nrm, sm, part);
    const double nq = sqrt(nrm[0]);
    if (!(nq > 1e-12 * sqrt(orig))) {  // the same decision in every CTA of the cluster
      if (threadIdx.x == 0 && rank == 0) atomicExch(err, 2);
      return;
    }
    const double inv = 1.0 / nq;
    for (int e = e0 + threadIdx.x; e < e1; e += NT) q[e] = make_double2(q[e].x * inv, q[e].y * inv);
    __syncthreads();
  }
}

int launch_block_gs(const Agg& g, const double2* cand, double2* P, int* err, cudaStream_t st) {
  if (g.nv > kGsMaxNv) return -1;
  block_gs_kernel<256><<<g.Vc * 2 * kGsCluster, 256, 0, st>>>(g, cand, P, err);
  return launched() ? 0 : -1;
}

// Column j of P (j = chi' nv + k') as a level-l field (chunk g.q): the k'-th
// orthonormal vector on its chirality chi' half, zero on the other half.
template <typename TP>
__global__ void p_column_kernel(const Agg g, const TP* P, int j0, TP* vbase) {
  const size_t tot = (size_t)g.ncomp * g.V;
  const int j = j0 + blockIdx.y;
  TP* v = vbase + (size_t)blockIdx.y * tot;
  const int chi = j / g.nv, k = j - chi * g.nv;
  const int len = g.nhalf * g.bsites;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    // element e of the field (chunk g.q): component c of site `site`
    int c, site;
    if (g.q == 4) {
      c = (int)((e / ((size_t)4 * g.V)) * 4 + (e & 3));
      site = (int)((e >> 2) % g.V);
    } else {
      c = (int)(e / g.V);
      site = (int)(e % g.V);
    }
    TP val;
    stc(&val, 0, zero<double>());
    if (c / g.nhalf == chi) {
      int cf[4], cb[4], cl[4];
      site_coords(site, g.L, cf);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        cb[m] = cf[m] / g.blk[m];
        cl[m] = cf[m] - cb[m] * g.blk[m];
      }
      const int B = site_index(cb, g.Lc), s = site_index(cl, g.blk);
      val = P[(((size_t)B * 2 + chi) * g.nv + k) * len + (size_t)(c - chi * g.nhalf) * g.bsites + s];
    }
    v[e] = val;
  }
}

int launch_p_column(int prec, const Agg& g, const void* P, int j0, int ncols, void* v, cudaStream_t st) {
  size_t tot = (size_t)g.ncomp * g.V;
  size_t b = (tot + 255) / 256;
  if (b > 8192) b = 8192;
  if (prec == 0)
    p_column_kernel<double2><<<dim3((unsigned)b, ncols), 256, 0, st>>>(g, (const double2*)P, j0, (double2*)v);
  else if (prec == 1)
    p_column_kernel<float2><<<dim3((unsigned)b, ncols), 256, 0, st>>>(g, (const float2*)P, j0, (float2*)v);
  else
    return -1;
  return launched() ? 0 : -1;
}

// ------------------------------------------------------------------ Galerkin build
// h = A_d(n) v(n + e_d) on every site of aggregate B into sm_h[c][s], in the
// arithmetic of the field's storage (FP64 for the plain hierarchy, FP32 for
// the mixed one).
template <typename TV, typename TL, int NL>
struct WilsonHopOp {
  typedef typename Store<TV>::R R;
  const TL* U;  // links, layout of wilson_hop.cuh
  double mass;
  __device__ void apply(const Agg& g, int B, int d, const TV* v, cx<R>* h, int nt) const {
    for (int s = threadIdx.x; s < g.bsites; s += nt) {
      const int n = agg_site2(g, B, s);
      cx<R> acc[4][3];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[sp][a] = zero<R>();
      if (d == 0) {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int a = 0; a < 3; ++a) acc[sp][a] = (R)(4.0 + mass) * ldc<R>(v, fidx(sp * 3 + a, n, g.V));
      } else {
        int c[4];
        site_coords(n, g.L, c);
        const int nb = neighbor(c, g.L, d);
        const int mu = (d - 1) >> 1;
        const bool fwd = d & 1;
        Link<R> u;
        load_link<R, TL, NL>(u, U, mu, g.V, fwd ? n : nb);
        switch (d) {
          case 1: hop<0, true>(acc, v, g.V, nb, u); break;
          case 2: hop<0, false>(acc, v, g.V, nb, u); break;
          case 3: hop<1, true>(acc, v, g.V, nb, u); break;
          case 4: hop<1, false>(acc, v, g.V, nb, u); break;
          case 5: hop<2, true>(acc, v, g.V, nb, u); break;
          case 6: hop<2, false>(acc, v, g.V, nb, u); break;
          case 7: hop<3, true>(acc, v, g.V, nb, u); break;
          default: hop<3, false>(acc, v, g.V, nb, u); break;
        }
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int a = 0; a < 3; ++a) acc[sp][a] = (R)(-0.5) * acc[sp][a];
      }
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) h[(sp * 3 + a) * g.bsites + s] = acc[sp][a];
    }
  }
};

template <typename TV>
struct StencilHopOp {
  typedef typename Store<TV>::R R;
  const TV* C;  // [9][n][n][V] of the level being coarsened
  __device__ void apply(const Agg& g, int B, int d, const TV* v, cx<R>* h, int nt) const {
    const int n = g.ncomp;
    for (int e = threadIdx.x; e < n * g.bsites; e += nt) {
      const int i = e / g.bsites, s = e - i * g.bsites;
      const int site = agg_site2(g, B, s);
      int c[4];
      site_coords(site, g.L, c);
      const int nb = neighbor(c, g.L, d);
      cx<R> acc = zero<R>();
      const TV* row = C + ((size_t)(d * n + i) * n) * g.V + site;
      for (int j = 0; j < n; ++j) acc = cfma(ldc<R>(row, (size_t)j * g.V), ldc<R>(v, (size_t)j * g.V + nb), acc);
      h[e] = acc;
    }
  }
};

// Does the hop d from aggregate-local site s leave the aggregate?
__device__ __forceinline__ bool crosses(const Agg& g, int s, int d) {
  if (d == 0) return false;
  int cl[4];
  site_coords(s, g.blk, cl);
  const int mu = (d - 1) >> 1;
  return (d & 1) ? (cl[mu] == g.blk[mu] - 1) : (cl[mu] == 0);
}

template <typename Op, typename TP, int NT>
__global__ void __launch_bounds__(NT) galerkin_kernel(const Agg g, Op op, const TP* vbase, const TP* P, int j0,
                                                      double2* Cout) {
  typedef typename Store<TP>::R R;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* h = (cx<R>*)smem_raw;                        // [ncomp][bsites]
  cx<R>* acc0 = h + (size_t)g.ncomp * g.bsites;       // [2 nv]
  const int j = j0 + blockIdx.y;
  const TP* vj = vbase + (size_t)blockIdx.y * g.ncomp * g.V;
  const int B = blockIdx.x;
  const int nc = 2 * g.nv;  // coarse components
  const int len = g.nhalf * g.bsites;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < nc; i += NT) acc0[i] = zero<R>();
  __syncthreads();
  for (int d = 0; d < 9; ++d) {
    op.apply(g, B, d, vj, h, NT);
    __syncthreads();
    for (int row = warp; row < nc; row += NT / 32) {
      const int chi = row / g.nv;
      const TP* pr = P + ((size_t)B * 2 * g.nv + row) * len;
      const cx<R>* hv = h + (size_t)chi * len;
      cx<R> in = zero<R>(), out = zero<R>();
      // site-major: the site's crossing test once, its nhalf components' loads in flight together
      for (int s = lane; s < g.bsites; s += 32) {
        cx<R> t = zero<R>();
#pragma unroll 6
        for (int c = 0; c < g.nhalf; ++c) {
          const int e = c * g.bsites + s;
          t = t + cmul_conj(ldc<R>(pr, e), hv[e]);
        }
        if (crosses(g, s, d))
          out = out + t;
        else
          in = in + t;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        in.re += __shfl_down_sync(0xffffffffu, in.re, o);
        in.im += __shfl_down_sync(0xffffffffu, in.im, o);
        out.re += __shfl_down_sync(0xffffffffu, out.re, o);
        out.im += __shfl_down_sync(0xffffffffu, out.im, o);
      }
      if (lane == 0) {
        acc0[row] = acc0[row] + in;
        if (d > 0) Cout[((size_t)(d * nc + row) * nc + j) * g.Vc + B] = make_double2(out.re, out.im);
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nc; i += NT)
    Cout[((size_t)(0 * nc + i) * nc + j) * g.Vc + B] = make_double2(acc0[i].re, acc0[i].im);
}

template <typename Op, typename TP>
static int galerkin_t(const Agg& g, const Op& op, const void* vj, const void* P, int j0, int ncols, double2* Cout,
                      cudaStream_t st) {
  typedef typename Store<TP>::R R;
  constexpr int NT = 256;
  const size_t sm = ((size_t)g.ncomp * g.bsites + 2 * g.nv) * sizeof(cx<R>);
  if (sm > kGalerkinSmemMax) return -1;  // mg_setup rejects such blocks up front
  if (sm > 48 * 1024)
    allow_big_smem(galerkin_kernel<Op, TP, NT>);
  galerkin_kernel<Op, TP, NT><<<dim3(g.Vc, ncols), NT, sm, st>>>(g, op, (const TP*)vj, (const TP*)P, j0, Cout);
  return launched() ? 0 : -1;
}

// prec 0: FP64 links (18 reals), P and fields; prec 1: FP32 links (12 reals), P and fields.
int launch_galerkin_wilson(int prec, const Agg& g, const void* links, double mass, const void* vj, const void* P,
                           int j0, int ncols, double2* Cout, cudaStream_t st) {
  if (prec == 0) {
    WilsonHopOp<double2, double2, 9> op;
    op.U = (const double2*)links;
    op.mass = mass;
    return galerkin_t<decltype(op), double2>(g, op, vj, P, j0, ncols, Cout, st);
  }
  if (prec == 1) {
    WilsonHopOp<float2, float2, 6> op;
    op.U = (const float2*)links;
    op.mass = mass;
    return galerkin_t<decltype(op), float2>(g, op, vj, P, j0, ncols, Cout, st);
  }
  return -1;
}

int launch_galerkin_stencil(int prec, const Agg& g, const void* Cfine, const void* vj, const void* P, int j0,
                            int ncols, double2* Cout, cudaStream_t st) {
  if (prec == 0) {
    StencilHopOp<double2> op;
    op.C = (const double2*)Cfine;
    return galerkin_t<decltype(op), double2>(g, op, vj, P, j0, ncols, Cout, st);
  }
  if (prec == 1) {
    StencilHopOp<float2> op;
    op.C = (const float2*)Cfine;
    return galerkin_t<decltype(op), float2>(g, op, vj, P, j0, ncols, Cout, st);
  }
  return -1;
}

}  // namespace wmg
