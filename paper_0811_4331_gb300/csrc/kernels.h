// Host-side launch interface shared by the translation units of the library.
// Precision codes: 0 = FP64, 1 = FP32, 2 = FP16, 3 = BF16 (storage of complex
// elements); arithmetic is FP64 for code 0 and FP32 otherwise.  Every
// launcher returns 0 on success and -1 on an invalid argument or launch error.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace wmg {

// Largest lattice (sites): the level-0 kernels index within one field and the
// links in 32-bit arithmetic (36 V < 2^32).
constexpr long long kMaxSites = 1LL << 26;

// ------------------------------------------------------------------ fine stencil
struct DslashCall {
  int prec;
  const void* in;
  void* out;
  const void* y;      // optional: out += c * y
  const void* z;      // optional: reduce <out|z>, ||out||^2 into red.result
  const void* links;  // packed links of precision prec
  int L[4];
  double a, b, c;     // out = a in + b Hop(in) + c y
  int nrhs;
  RedArgs red;        // lane = right-hand side, 3 values
  int variant = -1;   // launch shape (wilson_variants), -1 = default
  const double* adiag = nullptr;  // per right-hand side: a is a * adiag[r] (a mass per right-hand side)
};
int launch_wilson(const DslashCall& d, cudaStream_t st);
// MR step fused with the previous step's update: with c = omega
// dots[0..1] / dots[2] per right-hand side (stride dstride),
//   x = xin + c u (xin null: 0; u null: d.in),  rout = d.in - c pprev,
//   d.out = d.a rout + d.b Hop(rout),  <d.out|rout>, ||d.out||^2 into d.red.
// d.in, pprev, rout and d.out distinct; x may equal xin.
int launch_wilson_mr(const DslashCall& d, const void* pprev, const void* u, const void* xin, void* x, void* rout,
                     const double* dots, int dstride, double omega, cudaStream_t st);
int wilson_variants(int prec, bool dots, int nrhs, int V);
int wilson_blocks(int V);
int launch_pack_links(int prec, const void* ext, void* out, int V, cudaStream_t st);
// *worst = max over links of |U U^+ - 1|, |det U - 1| as float bits (caller zeroes it first).
int launch_su3_check(const void* ext, int V, unsigned* worst, cudaStream_t st);

// Even-odd stencil on half-lattice fields [nrhs][3][V/2][4] (every extent
// even): out_p = a x_p + b H_{p,1-p} in_{1-p} + c y_p, H the hopping term of
// D = (4 + m) - H / 2; links in the layout of wilson_hop.cuh with the sites
// parity-major (launch_eo_links).
struct EoCall {
  int prec;
  int parity;  // of out
  const void* x;  // may be null
  const void* in;
  const void* y;  // may be null
  const void* z;  // optional: reduce <out|z>, ||out||^2 per right-hand side into red
  void* out;
  const void* links;
  int L[4];
  double a, b, c;
  int nrhs;
  RedArgs red;
};
int launch_wilson_eo(const EoCall& d, cudaStream_t st);
int eo_blocks(int V);
// full rows of V elements (elem_bytes each: 4, 8, 16, 32 or 64) -> even and
// odd rows of V/2 at stride hstride.  A chunked level-0 field is 3 nrhs rows
// of 4-complex chunks.
int launch_eo_split(size_t elem_bytes, const void* full, void* even, void* odd, const int L[4], size_t rows,
                    size_t hstride, cudaStream_t st);
// Packed links of precision prec -> the same links with the sites parity-major.
int launch_eo_links(int prec, const void* links, void* out, const int L[4], cudaStream_t st);
// full = (add ? full : 0) + merge(even, odd), rows of V / V/2 four-complex
// chunks (3 nrhs rows for a level-0 field); a null half is zero.
int launch_eo_merge(int prec, const void* even, const void* odd, void* full, const int L[4], size_t rows, int add,
                    cudaStream_t st);

// ------------------------------------------------------------------ vectors
// Every vector kernel works on nrhs vectors of n complex elements each,
// right-hand side r at offset r * n.  Grid sizes are a pure function of n.
int vec_blocks(size_t n);
int red_blocks(size_t n);
const int kVecThreads = 256;
const int kMaxVecBlocks = 1216;  // upper bound of vector-kernel grids (8 per SM, 152 SMs on GB300); sizes partial buffers

// x_out = (x_in or 0) + alpha u;  r_out = r_in - alpha p, with per-rhs
// alpha = omega * (d[0] + i d[1]) / d[2] read from dots[rhs * dstride]
// (alpha = 0 when d[2] is 0 or not finite).  Optional reduction of
// ||r_out||^2 into red (lane rhs, 1 value).
struct MrUpdate {
  int prec;
  size_t n;
  int nrhs;
  void* x_out;
  const void* x_in;  // may be null (zero) or equal to x_out
  const void* u;
  void* r_out;
  const void* r_in;  // may equal r_out
  const void* p;
  const double* dots;
  int dstride;
  double omega;
  RedArgs red;  // red.result == null: no reduction
};
int launch_mr_update(const MrUpdate& m, cudaStream_t st);

// <a|b>, ||a||^2, ||b||^2 per rhs into red (4 values: re, im, |a|^2, |b|^2).
int launch_dot(int prec, size_t n, int nrhs, const void* a, const void* b, RedArgs red, cudaStream_t st);

// Classical Gram-Schmidt pieces for flexible GCR.
// Basis vector j of rhs r at base + j * jstride + r * n (elements).
// multidot: beta_j = <W_j|w> for j < k -> result[(r * kmax + j) * 2 + {0,1}] (red.stride
// ignored; result holds kmax complex per rhs).  W must hold ceil(k / 8) * 8 vectors.
int launch_multidot(int prec, size_t n, int nrhs, int k, int kmax, const void* W, size_t jstride,
                    const void* w, RedArgs red, cudaStream_t st, const double* pre = nullptr,
                    const double* post = nullptr, int cstride = 0);
// out = sum_t c[t] x[t] (FP64, complex host coefficients, null x[t] = unused
// term); with w, <w|out> and ||out||^2 are reduced into red (lane 0).
struct LinComb {
  double2* out;
  const double2* x[3];
  double2 c[3];
  const double2* w;
};
int launch_lincomb(size_t n, const LinComb& L, RedArgs red, cudaStream_t st);
// Outer GCR with a deferred solution update (A Z = W H, x += Z H^-1 alpha at
// the end of a cycle).  gs_update: w -= sum_j beta_j W_j with fused <w|r>,
// ||w||^2 and H[:, hk] += beta; pre/post/cstride as for the multi-dot (a
// second pass runs only where the first removed more than half of ||w||^2).
int launch_gs_update(int prec, size_t n, int nrhs, int k, int kmax, const double* beta, const void* W, size_t jstride,
                     void* w, const void* r, RedArgs red, double2* H, int hk, const double* pre, const double* post,
                     int cstride, cudaStream_t st);
// w /= ||w||, alpha_k = <w|r>, r -= alpha_k w with fused ||r||^2; stores H[k][k], alpha_k.
int launch_gcr_step(int prec, size_t n, int nrhs, const double* dots, int dstride, void* w, void* r, RedArgs red,
                    double2* H, double2* alpha, int k, int kmax, cudaStream_t st);
// y = H^-1 alpha (upper triangular, per right-hand side).
int launch_back_substitute(int nrhs, int k, int kmax, const double2* H, const double2* alpha, double2* y,
                           cudaStream_t st);
// x += sum_j y_j Z_j.
int launch_zcombine(int zprec, int xprec, size_t n, int nrhs, int k, int kmax, const double2* y, const void* Z,
                    size_t jstride, void* x, cudaStream_t st);
// w -= sum_j beta_j W_j, z -= sum_j beta_j Z_j (beta from multidot result);
// then reduce ||w||^2 and <w|r> per rhs into red2 (3 values: re, im, |w|^2).
int launch_multiaxpy(int prec, size_t n, int nrhs, int k, int kmax, const double* beta, const void* W,
                     const void* Zb, size_t jstride, void* w, void* z, const void* r, RedArgs red2,
                     cudaStream_t st);
// GCR step from dots = (<w|r>, ||w||^2) per rhs: w /= |w|, z /= |w|,
// a = <w|r> / |w|, x += a z, r -= a w; reduce ||r||^2 into red (1 value).
// x may have a different precision (xprec) than the others.
int launch_gcr_update(int prec, int xprec, size_t n, int nrhs, const double* dots, int dstride, void* w,
                      void* z, void* x, void* r, RedArgs red, cudaStream_t st);

// out = scale * in (+ out if accumulate), converting precision.  scale =
// s0 * (slot ? pow(slot[rhs * sstride], sexp) : 1).
int launch_convert(int pin, int pout, size_t n, int nrhs, const void* in, void* out, double s0,
                   const double* slot, int sstride, double sexp, int accumulate, cudaStream_t st);

// External [nrhs][V][ncomp] FP64 complex <-> internal fields of precision
// prec and chunk q (4: level 0, 1: coarse levels; see fidx_q).
int launch_ext_to_int(int prec, int ncomp, int q, int V, int nrhs, const void* ext, void* internal, cudaStream_t st);
int launch_int_to_ext(int prec, int ncomp, int q, int V, int nrhs, const void* internal, void* ext, cudaStream_t st);

// out = gamma5 in on FP64 level-0 fields of V sites (chunked layout; in == out allowed).
int launch_gamma5(size_t V, int nrhs, const void* in, void* out, cudaStream_t st);

// Counter-based Gaussian start vectors (SplitMix64 + Box-Muller), FP64
// internal fields of chunk q, nv of them; element (k, site, comp) is stream
// element k V ncomp + site ncomp + comp of stream `seed`.
int launch_gaussian_starts(uint64_t seed, int nv, int ncomp, int q, int V, void* out, cudaStream_t st);

// ------------------------------------------------------------------ coarse levels
struct CoarseCall {
  int prec;
  const void* C;  // [9][ncomp][ncomp][V]
  const void* in;
  void* out;
  const void* y;  // optional: out = a A in + c y
  const void* z;  // optional dots <out|z>, ||out||^2
  int L[4];
  int ncomp;
  double a, c;
  int nrhs;
  RedArgs red;
  const double* shift = nullptr;  // per right-hand side: out = a (A + shift[r] 1) in + c y
};
int launch_coarse_apply(const CoarseCall& k, cudaStream_t st);
int coarse_blocks(int ncomp, int V);

// Tensor-core coarse stencil (BF16 mma.sync, FP32 accumulation) for R <= 64
// right-hand sides of storage prec (1 = FP32, 3 = BF16): out = a A in + c y2.
size_t mma_pack_bytes(int n, int V);
int launch_mma_pack(const double2* C, int n, int V, void* out, cudaStream_t st);
// variant >= 0 picks one of coarse_mma_variants(R) launch shapes (right-hand
// sides split over CTAs); every shape gives bit-identical results.
int launch_coarse_mma(int prec, const void* Cf, const void* in, void* out, const void* y2, const int L[4], int n, int R,
                      double a, double c, cudaStream_t st, int variant = -1, const double* shift = nullptr);
int coarse_mma_variants(int R);

// Aggregation of level l (fine side) into level l+1 (coarse side).
struct Agg {
  int L[4];
  int V;
  int ncomp;
  int q;  // chunk of the fine-side fields (4 on level 0, 1 on coarse levels)
  int nhalf;
  int nv;
  int blk[4];
  int bsites;
  int Lc[4];
  int Vc;
};
int launch_restrict(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                    cudaStream_t st, int variant = -1);
int launch_prolong(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                   cudaStream_t st, int variant = -1);
// Tensor-core transfers for 2..64 right-hand sides with 16-bit P (nv <= 64,
// nv / 16 rounded up in {1, 2, 4}); launch_restrict / launch_prolong pick them.
bool transfer_mma_ok(const Agg& g, int nrhs);
int launch_restrict_mma(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                        cudaStream_t st, int variant = -1);
int launch_prolong_mma(int pin, int pP, int pout, const Agg& g, const void* P, const void* in, void* out, int nrhs,
                       cudaStream_t st, int variant = -1);
// Launch shapes of the tensor-core transfers (right-hand sides split over CTAs; bit-identical results).
int transfer_mma_variants(int nrhs);

// C_0(B) += delta 1 on a coarse stencil [9][n][n][V] (FP64).
int launch_diag_shift(double2* C, int n, int V, double delta, cudaStream_t st);

// Coarsest level: dense inverse (Gauss-Jordan, partial pivoting) of an FP64
// stencil operator in precision prec (0 or 1); aug is [N][2N] of precision
// prec, scratch holds dense_inverse_scratch_bytes(prec, N), inv is [N][N];
// *err = 1 on a zero pivot.  N + 2 launches.
int dense_inverse(int prec, const double2* C, const int L[4], int n, void* aug, void* scratch, int* err, void* inv,
                  cudaStream_t st);
size_t dense_inverse_scratch_bytes(int prec, int N);
// The same for `batch` independent matrices (C[z] -> inv[z], host arrays of
// device pointers) sharing every elimination launch; aug holds batch N x 2N
// matrices, scratch batch x dense_inverse_scratch_bytes(prec, N), err batch
// flags.
// With blk (gjb_scratch_bytes(N, element size, batch) bytes, 0 = not
// available for this N) the elimination runs in panels and rank-64 blocks
// (blocked form).  *launches (optional) = the kernels it launched.
int dense_inverse_batch(int prec, const double2* const* C, const int L[4], int n, int batch, void* aug, void* scratch,
                        int* err, void* const* inv, void* blk, cudaStream_t st, long long* launches);
size_t gjb_scratch_bytes(int N, size_t eb, int batch);
// y = inv x (+ y if acc); (matrix, in, out) precisions (0,0,0), (1,0,0), (1,1,1).
// With scratch (dense_matvec_scratch_bytes(N), tickets zeroed once) 4..64
// right-hand sides run as one tiled product; otherwise one warp per row and
// right-hand side.  midx (device, optional): right-hand side r uses matrix
// midx[r] of inv = [count][N][N] (always the row-per-warp form).
int launch_dense_matvec(int pm, int pin, int pout, int N, const void* inv, const void* x, void* y, int nrhs,
                        int acc, cudaStream_t st, void* scratch, const int* midx = nullptr);
size_t dense_matvec_scratch_bytes(int N);

// Setup: blockwise Gram-Schmidt (err = 2 on rank loss), prolongator
// columns as fields, Galerkin coarse stencil column j.
int launch_block_gs(const Agg& g, const double2* cand, double2* P, int* err, cudaStream_t st);
// Columns j0 .. j0 + ncols - 1 at v + (j - j0) * ncomp * V, precision prec (0 or 1) of P and v.
int launch_p_column(int prec, const Agg& g, const void* P, int j0, int ncols, void* v, cudaStream_t st);
// Galerkin columns in the arithmetic of `prec` (0: FP64 inputs, 1: FP32 inputs); output always FP64 storage.
// Shared memory of one Galerkin CTA: a block of the P column (ncomp x bsites)
// plus 2 nv coefficients, complex in the setup's precision (0 FP64, 1 FP32).
constexpr size_t kGalerkinSmemMax = 200 * 1024;
inline size_t galerkin_smem_bytes(int prec, int ncomp, int bsites, int nv) {
  return ((size_t)ncomp * bsites + 2 * (size_t)nv) * (prec == 0 ? 16 : 8);
}
int launch_galerkin_wilson(int prec, const Agg& g, const void* links, double mass, const void* vj, const void* P,
                           int j0, int ncols, double2* Cout, cudaStream_t st);
int launch_galerkin_stencil(int prec, const Agg& g, const void* Cfine, const void* vj, const void* P, int j0,
                            int ncols, double2* Cout, cudaStream_t st);

}  // namespace wmg
