// C ABI of the library and the host-side orchestration of the solver:
// setup of the multigrid hierarchy (Sec. 2 adaptive steps, Eq. 2.3, Sec. 3),
// the modified V(2,2) cycle with the alpha-damped coarse-grid correction
// (Sec. 3 Eq. 3.5, Sec. 5) and flexible GCR(50) (Sec. 5), plain FP64 or
// mixed precision with FP64 reliable updates.  All arithmetic runs in the
// kernels of this library; the host only sequences launches and reads the
// residual norms that decide when to stop.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "handle.h"

namespace wmg {

static thread_local std::string g_err = "";
void set_error(const std::string& msg) { g_err = msg; }
// kernels launched by this library since it was loaded (all handles, all threads)
static unsigned long long g_launches = 0;
// profiler mask that new handles start with (mg_profile(NULL, mask))
static unsigned g_default_prof_mask = 0;
// the same count for the calling thread only (what a graph capture on this thread recorded)
static thread_local unsigned long long tl_launches = 0;
inline void count_launches(unsigned long long n) {
  __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED);
  tl_launches += n;
}

}  // namespace wmg

using namespace wmg;

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string(#x) + ": " + cudaGetErrorString(e_));                      \
      return MG_ECUDA;                                                                 \
    }                                                                                  \
  } while (0)
#define LK(x)                                                                          \
  do {                                                                                 \
    count_launches(1);                                                                 \
    if ((x) != 0) {                                                                    \
      cudaError_t e_ = cudaGetLastError();                                             \
      if (e_ == cudaSuccess) e_ = take_launch_error();                                 \
      set_error(std::string("launch failed: ") + #x + ": " + cudaGetErrorString(e_));  \
      return e_ == cudaSuccess ? MG_EINVAL : MG_ECUDA;                                 \
    }                                                                                  \
  } while (0)
#define RET(x)                      \
  do {                              \
    int r_ = (x);                   \
    if (r_ != MG_OK) return r_;     \
  } while (0)

extern "C" unsigned long long mg_launch_count(void);

namespace {

// Result-slot map (doubles) inside the reducer's slot array.
const int kMaxRhs = 64;
const int kMaxBasis = 64;  // GCR restart length cap (multiple of 8)
inline size_t slot_level(int l) { return (size_t)l * 4 * kMaxRhs; }
inline size_t slot_gcr_wr() { return slot_level(MG_MAX_LEVELS); }
inline size_t slot_gcr_rn() { return slot_gcr_wr() + 4 * kMaxRhs; }
inline size_t slot_gcr_bn() { return slot_gcr_rn() + 4 * kMaxRhs; }
inline size_t slot_misc() { return slot_gcr_bn() + 4 * kMaxRhs; }
inline size_t slot_beta() { return slot_misc() + 4 * kMaxRhs; }
// inner GCR of the coarse correction of level l: dots, residual norms, betas (8 per rhs)
inline size_t slot_inner(int l) { return slot_beta() + (size_t)2 * kMaxBasis * kMaxRhs + (size_t)l * 24 * kMaxRhs; }
inline size_t slot_gcr_pre() { return slot_inner(MG_MAX_LEVELS); }  // <w|r>, ||w||^2 before Gram-Schmidt
inline size_t slot_total() { return slot_gcr_pre() + 4 * kMaxRhs; }
const int kInnerBasis = 8;

enum { WV_E, WV_RES, WV_P, WV_XC, WV_AXC, WV_RC, WV_EC, WV_T, WV_DT, WV_IN, WV_A, WV_B, WV_KW, WV_KZ, WV_PR, WV_PE, WV_EOA, WV_EOB, WV_EOC, WV_COUNT };

int prec_of(const mg_handle* h, int l) {
  if (!h->p.mixed) return MG_F64;
  const int L = h->p.n_levels;  // not lev.size(): during setup the levels below l may not exist yet
  if (l == 0) return h->p.fine_prec;
  if (l == L - 1) return MG_F32;  // coarsest vectors; the inverse stays FP64
  return h->p.coarse_prec;
}

Agg agg_of(const Level& a) {
  Agg g;
  for (int m = 0; m < 4; ++m) {
    g.L[m] = a.L[m];
    g.blk[m] = a.blk[m];
    g.Lc[m] = a.Lc[m];
  }
  g.V = a.V;
  g.ncomp = a.ncomp;
  g.q = a.q;
  g.nhalf = a.nhalf;
  g.nv = a.nv;
  g.bsites = a.bsites;
  g.Vc = a.Vc;
  return g;
}

size_t bytes_of(int prec) { return prec == MG_F64 ? 16 : (prec == MG_F32 ? 8 : 4); }

int check_prec(int prec) { return (prec >= 0 && prec <= 3) ? MG_OK : MG_EINVAL; }

void* work(mg_handle* h, int l, int prec, int idx, int nrhs, int count = 1) {
  if ((int)h->work.size() <= l) h->work.resize(l + 1);
  auto& byprec = h->work[l];
  if (byprec.empty()) byprec.resize(4);
  auto& vecs = byprec[prec];
  if ((int)vecs.size() <= idx) vecs.resize(idx + 1);
  if (!vecs[idx]) vecs[idx].reset(new DevBuf());
  const size_t need = h->lev[l]->n() * (size_t)nrhs * bytes_of(prec) * (size_t)count;
  if (need > vecs[idx]->bytes || !vecs[idx]->p) {
    if (h->capturing) return nullptr;  // never allocate inside a capture
    ++h->buf_gen;
  }
  if (!vecs[idx]->ensure(need)) return nullptr;
  return vecs[idx]->p;
}

int ensure_reducer(mg_handle* h, int nrhs) {
  if (nrhs > kMaxRhs) {
    set_error("nrhs above the library limit of 64");
    return MG_EINVAL;
  }
  size_t need = (size_t)kMaxVecBlocks * 16 * ((kMaxBasis / 8) * (size_t)nrhs + 1);
  for (auto& lp : h->lev) {
    const Level& a = *lp;
    size_t b = a.q == 4 ? (size_t)wilson_blocks(a.V) : (size_t)coarse_blocks(a.ncomp, a.V);  // level 0: the stencil
    need = std::max(need, b * 3 * (size_t)nrhs);
  }
  if (need <= h->red.max_partials && h->red.nslots) return MG_OK;
  if (h->capturing) return MG_EINVAL;
  cudaStreamSynchronize(h->st);
  ++h->buf_gen;
  if (!h->red.init(need, (int)slot_total(), 4096)) {
    set_error("out of device memory for reduction scratch");
    return MG_ENOMEM;
  }
  return MG_OK;
}

// Per-launch event profiler (mg_profile): brackets each launch of a selected
// kernel class with a pair of events on the handle's stream.
// Event pair around the launches of one scope, with the scope's algorithmic
// bytes (each operand read or written once; 0 where not counted).
struct Prof {
  mg_handle* h;
  bool on;
  size_t idx = 0;
  int key;
  double bytes;
  Prof(mg_handle* hh, int cls, int prec, double nbytes = 0.0)
      : h(hh), on(((hh->prof_mask >> cls) & 1u) && !hh->capturing), key(cls * 4 + prec), bytes(nbytes) {
    if (!on) return;
    while (h->prof_used + 2 > h->prof_pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        on = false;
        return;
      }
      h->prof_pool.push_back(e);
    }
    idx = h->prof_used;
    h->prof_used += 2;
    cudaEventRecord(h->prof_pool[idx], h->st);
  }
  ~Prof() {
    if (!on) return;
    cudaEventRecord(h->prof_pool[idx + 1], h->st);
    h->prof_marks.push_back({key, idx, bytes});
  }
};

// ------------------------------------------------------------------ launch-shape tuner
// Process-wide choice of the fastest launch shape for each (kernel, precision,
// sizes, right-hand sides).  The candidate shapes of every tuned kernel give
// bit-identical results (they only regroup right-hand sides or sites over
// CTAs), so tuning changes speed, never numbers.  On the first launch of a
// key outside graph capture each shape runs once to warm up and kTuneReps
// times between two events on the handle's stream, writing scratch outputs
// only; a shape whose launch fails is skipped.  Mode 0 turns tuning off
// (default shapes), 1 tunes, and 3 / 4 force the last / first shape of every
// key (to check that all shapes agree).
struct TuneEntry {
  int variant;
  std::vector<float> us;
};
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune;
int g_tune_mode = 1;
const int kTuneReps = 3;

template <class F>
int tuned(mg_handle* h, const std::string& key, int nvar, F&& run) {
  if (nvar <= 1 || g_tune_mode == 0) return -1;
  if (g_tune_mode == 3) return nvar - 1;
  if (g_tune_mode == 4) return 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it != g_tune.end()) return it->second.variant;
  if (h->capturing) return -1;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1;
  }
  std::vector<float> us(nvar, -1.0f);
  int best = -1;
  float bt = 0.0f;
  for (int v = 0; v < nvar; ++v) {
    if (run(v) != 0) {
      cudaGetLastError();
      continue;
    }
    bool ok = cudaEventRecord(e0, h->st) == cudaSuccess;
    for (int r = 0; r < kTuneReps && ok; ++r) ok = run(v) == 0;
    ok = ok && cudaEventRecord(e1, h->st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.0f;
    if (!ok || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    us[v] = ms * 1000.0f / kTuneReps;
    if (best < 0 || us[v] < bt) {
      best = v;
      bt = us[v];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_tune[key] = {best, us};
  count_launches((unsigned long long)nvar * (kTuneReps + 1));
  return best;
}

std::string tkey(const char* kernel, std::initializer_list<long long> v) {
  std::string k = kernel;
  for (long long x : v) k += "|" + std::to_string(x);
  return k;
}

// out = a_ * (A_l in) + c_ * y; optional dots <out|z>, ||out||^2 into slot.
int op_apply(mg_handle* h, int l, int prec, const void* in, void* out, const void* y, double a_, double c_,
             const void* z, size_t slot, int nrhs) {
  Level& a = *h->lev[l];
  if (l == 0) {
    if (!a.links[prec].p) {
      set_error("level-0 operator not stored in this precision");
      return MG_EINVAL;
    }
    DslashCall d;
    d.prec = prec;
    d.in = in;
    d.out = out;
    d.y = y;
    d.z = z;
    d.links = a.links[prec].p;
    for (int m = 0; m < 4; ++m) d.L[m] = a.L[m];
    d.a = h->mm_active ? a_ : a_ * (4.0 + h->mass);
    d.adiag = h->mm_active ? h->mm_adiag.as<double>() : nullptr;
    d.b = -0.5 * a_;
    d.c = c_;
    d.nrhs = nrhs;
    d.red = h->red.at(slot, 4);
    // spinor in and out per right-hand side, y and z where they are other vectors, links once
    const double sb = 12.0 * a.V * bytes_of(prec);
    const double lb = 4.0 * a.V * (prec == MG_F64 ? 9 : 6) * bytes_of(prec);
    {
      DevBuf scratch;
      d.variant = tuned(h, tkey("dslash", {prec, a.L[0], a.L[1], a.L[2], a.L[3], nrhs, y != nullptr, z != nullptr}),
                        wilson_variants(prec, z != nullptr, nrhs, a.V), [&](int v) {
                          if (!scratch.p && !scratch.ensure((size_t)a.n() * nrhs * bytes_of(prec))) return -1;
                          DslashCall t = d;
                          t.out = scratch.p;
                          t.variant = v;
                          return launch_wilson(t, h->st);
                        });
    }
    Prof pf(h, MG_K_DSLASH, prec, nrhs * sb * (2 + (y && y != in) + (z && z != in && z != y)) + lb);
    LK(launch_wilson(d, h->st));
  } else if (a.cop_mma.p && prec == MG_F32 && nrhs <= 64) {
    const double* mmshift = h->mm_active ? h->mm_shift.as<double>() : nullptr;
    // tensor cores: out = a_ A in + c_ y, then the dots in a separate deterministic pass
    const double vb = (double)a.n() * bytes_of(prec);
    {
      DevBuf scratch;
      const int var = tuned(h, tkey("coarse_mma", {prec, a.ncomp, a.V, nrhs}), coarse_mma_variants(nrhs), [&](int v) {
        if (!scratch.p && !scratch.ensure((size_t)vb * nrhs)) return -1;
        return launch_coarse_mma(prec, a.cop_mma.p, in, scratch.p, y, a.L, a.ncomp, nrhs, a_, c_, h->st, v, mmshift);
      });
      Prof pf(h, MG_K_COARSE, MG_BF16, (double)mma_pack_bytes(a.ncomp, a.V) + nrhs * vb * (2 + (y != nullptr)));
      LK(launch_coarse_mma(prec, a.cop_mma.p, in, out, y, a.L, a.ncomp, nrhs, a_, c_, h->st, var, mmshift));
    }
    if (z) {
      Prof pf(h, MG_K_VECTOR, prec, nrhs * vb * (z == out ? 1 : 2));
      LK(launch_dot(prec, a.n(), nrhs, out, z, h->red.at(slot, 4), h->st));
    }
  } else {
    if (!a.cop[prec].p) {
      set_error("coarse operator not stored in this precision");
      return MG_EINVAL;
    }
    CoarseCall k;
    k.prec = prec;
    k.C = a.cop[prec].p;
    k.in = in;
    k.out = out;
    k.y = y;
    k.z = z;
    for (int m = 0; m < 4; ++m) k.L[m] = a.L[m];
    k.ncomp = a.ncomp;
    k.a = a_;
    k.c = c_;
    k.nrhs = nrhs;
    k.red = h->red.at(slot, 4);
    k.shift = h->mm_active ? h->mm_shift.as<double>() : nullptr;
    const double vb = (double)a.n() * bytes_of(prec);
    Prof pf(h, MG_K_COARSE, prec,
            9.0 * a.ncomp * a.ncomp * a.V * bytes_of(prec) + nrhs * vb * (2 + (y && y != in) + (z && z != in && z != y)));
    LK(launch_coarse_apply(k, h->st));
  }
  return MG_OK;
}

int mr_update(mg_handle* h, int l, int prec, void* x_out, const void* x_in, const void* u, void* r_out,
              const void* r_in, const void* p, size_t slot, double omega, int nrhs, size_t n = 0) {
  MrUpdate m;
  m.prec = prec;
  m.n = n ? n : h->lev[l]->n();
  m.nrhs = nrhs;
  m.x_out = x_out;
  m.x_in = x_in;
  m.u = u;
  m.r_out = r_out;
  m.r_in = r_in;
  m.p = p;
  m.dots = h->red.slot(slot);
  m.dstride = 4;
  m.omega = omega;
  m.red = h->red.at(0, 0);
  m.red.result = nullptr;
  const int streams = 4 + (x_in != nullptr) + (r_in != r_out && r_in != u && r_in != p);  // u, p, r_in, x_out, r_out
  Prof pf(h, MG_K_VECTOR, prec, (double)streams * nrhs * m.n * bytes_of(prec));
  LK(launch_mr_update(m, h->st));
  return MG_OK;
}

// One level-0 MR step fused with the previous step's update (see
// launch_wilson_mr): x = xin + c u (u null: r; xin null: 0), rout = r - c p,
// pout = D rout with <pout|rout>, ||pout||^2 into slot; c = omega <p|r>/<p|p>
// is read from the same slot (every CTA reads it before the reduction's last
// CTA overwrites it).
int mr_fused(mg_handle* h, int prec, const void* r, const void* pv, const void* u, const void* xin, void* x,
             void* rout, void* pout, size_t slot, double omega, int nrhs) {
  Level& a = *h->lev[0];
  DslashCall d;
  d.prec = prec;
  d.in = r;
  d.out = pout;
  d.y = nullptr;
  d.z = nullptr;
  d.links = a.links[prec].p;
  for (int m = 0; m < 4; ++m) d.L[m] = a.L[m];
  d.a = 4.0 + h->mass;
  d.b = -0.5;
  d.c = 0.0;
  d.nrhs = nrhs;
  d.red = h->red.at(slot, 4);
  // r, p, u (if not r) and xin read; x, r' and p' written, per right-hand side; links once
  const double sb = 12.0 * a.V * bytes_of(prec);
  const double lb = 4.0 * a.V * (prec == MG_F64 ? 9 : 6) * bytes_of(prec);
  Prof pf(h, MG_K_DSLASH, prec, nrhs * sb * (5 + (u != nullptr) + (xin != nullptr)) + lb);
  LK(launch_wilson_mr(d, pv, u, xin, x, rout, h->red.slot(slot), 4, omega, h->st));
  return MG_OK;
}

// `steps` MR steps on A_l x = b continuing from (x, res): if x_zero the
// iterate is 0 and res is taken from b without an operator application.
int mr_steps(mg_handle* h, int l, int prec, const void* b, void* x, bool x_zero, void* res, int steps, int nrhs) {
  const size_t sl = slot_level(l);
  void* p = work(h, l, prec, WV_P, nrhs);
  if (!p) return MG_ENOMEM;
  const double omega = h->p.omega;
  if (steps == 0) {
    if (x_zero) {
      CK(cudaMemsetAsync(x, 0, h->lev[l]->n() * nrhs * bytes_of(prec), h->st));
      CK(cudaMemcpyAsync(res, b, h->lev[l]->n() * nrhs * bytes_of(prec), cudaMemcpyDeviceToDevice, h->st));
    }
    return MG_OK;
  }
  for (int s = 0; s < steps; ++s) {
    const void* rcur = (s == 0 && x_zero) ? b : res;
    RET(op_apply(h, l, prec, rcur, p, nullptr, 1.0, 0.0, rcur, sl, nrhs));
    RET(mr_update(h, l, prec, x, (s == 0 && x_zero) ? nullptr : x, rcur, res, rcur, p, sl, omega, nrhs));
  }
  return MG_OK;
}

// ------------------------------------------------------------------ even-odd (level 0)
// Half fields hold the V/2 sites of one parity, [nrhs][12][V/2] (see
// wilson_eo.cu); D = M - H/2 with M = 4 + m, H the hopping term.

// Level-0 links reordered parity-major in precision prec, built on first use.
int ensure_eo_links(mg_handle* h, int prec) {
  Level& f = *h->lev[0];
  if (f.links_eo[prec].p) return MG_OK;
  if (!f.links[prec].p) {
    set_error("level-0 operator not stored in this precision");
    return MG_EINVAL;
  }
  if (f.L[0] % 2 || f.L[1] % 2 || f.L[2] % 2 || f.L[3] % 2) {
    set_error("even-odd operators need every lattice extent even");
    return MG_EINVAL;
  }
  if (h->capturing) {
    set_error("even-odd links first needed inside a graph capture");
    return MG_EINVAL;
  }
  const size_t NL = prec == MG_F64 ? 9 : 6, eb = bytes_of(prec);
  if (!f.links_eo[prec].ensure((size_t)4 * NL * f.V * eb)) return MG_ENOMEM;
  char* base = (char*)f.links_eo[prec].p;
  LK(launch_eo_links(prec, f.links[prec].p, base, f.L, h->st));
  return MG_OK;
}

// out_p = a x_p + b H in_{1-p} + c y_p on half fields; with z, <out|z> and ||out||^2 into slot.
int eo_apply(mg_handle* h, int prec, int parity, const void* x, const void* in, const void* y, void* out, double a_,
             double b_, double c_, const void* z, size_t slot, int nrhs) {
  RET(ensure_eo_links(h, prec));
  Level& f = *h->lev[0];
  EoCall d;
  d.prec = prec;
  d.parity = parity;
  d.x = x;
  d.in = in;
  d.y = y;
  d.z = z;
  d.out = out;
  d.links = f.links_eo[prec].p;
  for (int m = 0; m < 4; ++m) d.L[m] = f.L[m];
  d.a = a_;
  d.b = b_;
  d.c = c_;
  d.nrhs = nrhs;
  d.red = h->red.at(slot, 4);
  // half spinors in, out, x, y and z where they are other vectors; every link once (forward hops read the
  // links of the output sites, backward hops those of the other parity)
  const double hb = 6.0 * f.V * bytes_of(prec);
  const double lb = 4.0 * f.V * (prec == MG_F64 ? 9 : 6) * bytes_of(prec);
  const int streams = 2 + (x != nullptr) + (y != nullptr) + (z && z != x && z != y);
  Prof pf(h, MG_K_DSLASH, prec, nrhs * hb * streams + lb);
  LK(launch_wilson_eo(d, h->st));
  return MG_OK;
}

// out = S in (y null) or y - S in, S = M - H_eo H_oe / (4 M) on even half fields; t is an odd half
// scratch; with z, <out|z> and ||out||^2 into slot.
int schur_op(mg_handle* h, int prec, const void* in, void* out, void* t, const void* y, const void* z, size_t slot,
             int nrhs) {
  const double M = 4.0 + h->mass;
  RET(eo_apply(h, prec, 1, nullptr, in, nullptr, t, 0.0, 1.0, 0.0, nullptr, 0, nrhs));
  if (y) return eo_apply(h, prec, 0, in, t, y, out, -M, 1.0 / (4.0 * M), 1.0, z, slot, nrhs);
  return eo_apply(h, prec, 0, in, t, nullptr, out, M, -1.0 / (4.0 * M), 0.0, z, slot, nrhs);
}

// Even-odd smoother on level 0 (not in the paper): e_e = `steps` under-relaxed
// MR steps (Sec. 3) on S e_e = r^_e = r_e + H_eo r_o / (2 M) from e_e = 0, and
// the odd sites solved exactly, e_o = (r_o + H_oe e_e / 2) / M.  e receives
// e_e + e_o (added to e when `add`), res the new residual r - D e, which is the
// Schur residual on even sites and 0 on odd ones.  res may alias r.
int eo_smooth(mg_handle* h, int prec, const void* r, void* e, bool add, void* res, int steps, int nrhs) {
  Level& f = *h->lev[0];
  const size_t nh = f.n() / 2, hb = nh * nrhs * bytes_of(prec);
  char* A = (char*)work(h, 0, prec, WV_EOA, nrhs);  // r_e | r_o
  char* B = (char*)work(h, 0, prec, WV_EOB, nrhs);  // Schur residual | odd scratch
  char* C = (char*)work(h, 0, prec, WV_EOC, nrhs);  // e_e | e_o
  char* Pv = (char*)work(h, 0, prec, WV_P, nrhs);   // S applied to the Schur residual
  if (!A || !B || !C || !Pv) return MG_ENOMEM;
  void *re = A, *ro = A + hb, *rs = B, *t = B + hb, *ee = C, *eo = C + hb;
  const double M = 4.0 + h->mass;
  const size_t sl = slot_level(0);
  {
    Prof pf(h, MG_K_VECTOR, prec, 2.0 * hb * 2);
    LK(launch_eo_split(4 * bytes_of(prec), r, re, ro, f.L, (size_t)3 * nrhs, (size_t)(f.V / 2), h->st));
  }
  RET(eo_apply(h, prec, 0, re, ro, nullptr, rs, 1.0, 1.0 / (2.0 * M), 0.0, nullptr, 0, nrhs));
  if (steps == 0) CK(cudaMemsetAsync(ee, 0, hb, h->st));
  for (int s = 0; s < steps; ++s) {
    RET(schur_op(h, prec, rs, Pv, t, nullptr, rs, sl, nrhs));
    RET(mr_update(h, 0, prec, ee, s == 0 ? nullptr : ee, rs, rs, rs, Pv, sl, h->p.omega, nrhs, nh));
  }
  RET(eo_apply(h, prec, 1, ro, ee, nullptr, eo, 1.0 / M, 1.0 / (2.0 * M), 0.0, nullptr, 0, nrhs));
  Prof pf(h, MG_K_VECTOR, prec, 2.0 * hb * (add ? 4 : 3));
  LK(launch_eo_merge(prec, ee, eo, e, f.L, (size_t)3 * nrhs, add ? 1 : 0, h->st));
  LK(launch_eo_merge(prec, rs, nullptr, res, f.L, (size_t)3 * nrhs, 0, h->st));
  return MG_OK;
}

// Site x candidate counts up to which the level-0 setup relaxation fuses each
// MR update into the next stencil launch (an 8^3 x 16 lattice with 20
// candidates is 163,840).
const size_t kFuseRelaxSites = 262144;

// Setup relaxation in FP32: steps between recomputations of the true residual.
const int kTrueResidualEvery = 25;

// Number of FP64 iterative-refinement steps of the mixed-precision coarsest solve.
const int kCoarsestRefine = 1;

// Exact solve on the coarsest level.  Plain: e = A^-1 r with the FP64
// inverse.  Mixed: with an FP64 inverse (coarsest_f64) e = A^-1 r in FP64
// from the converted input; with an FP32 inverse X the solve runs in FP64 as
// e = X r, then kCoarsestRefine times e += X (r - A e) with the FP64 stencil.
int coarsest_solve(mg_handle* h, int l, int prec, const void* r, void* e, int nrhs) {
  Level& a = *h->lev[l];
  // a mass per right-hand side: right-hand side r takes the inverse of its own mass
  const void* inv = h->mm_active ? h->mm_inv.p : a.inv.p;
  const int* midx = h->mm_active ? h->mm_idx.as<int>() : nullptr;
  const double mvb = (double)a.N() * a.N() * bytes_of(a.inv_prec) + 2.0 * nrhs * a.N() * 16;  // inverse once, x and y
  if (a.inv_prec == MG_F64 && prec == MG_F64) {
    Prof pf(h, MG_K_COARSEST, prec, mvb);
    LK(launch_dense_matvec(0, 0, 0, a.N(), inv, r, e, nrhs, 0, h->st, a.mm_scratch.p, midx));
    return MG_OK;
  }
  void* r64 = work(h, l, MG_F64, WV_A, nrhs);
  void* e64 = work(h, l, MG_F64, WV_B, nrhs);
  void* t64 = work(h, l, MG_F64, WV_T, nrhs);
  if (!r64 || !e64 || !t64) return MG_ENOMEM;
  const size_t n = a.n();
  {
    Prof pf(h, MG_K_VECTOR, prec);
    LK(launch_convert(prec, MG_F64, n, nrhs, r, r64, 1.0, nullptr, 0, 0.0, 0, h->st));
  }
  {
    Prof pf(h, MG_K_COARSEST, a.inv_prec, mvb);
    LK(launch_dense_matvec(a.inv_prec, 0, 0, a.N(), inv, r64, e64, nrhs, 0, h->st, a.mm_scratch.p, midx));
  }
  const int refine = a.inv_prec == MG_F64 ? 0 : kCoarsestRefine;
  for (int it = 0; it < refine; ++it) {
    RET(op_apply(h, l, MG_F64, e64, t64, r64, -1.0, 1.0, nullptr, 0, nrhs));
    Prof pf(h, MG_K_COARSEST, MG_F32, mvb + (double)nrhs * a.N() * 16);
    LK(launch_dense_matvec(a.inv_prec, 0, 0, a.N(), inv, t64, e64, nrhs, 1, h->st, a.mm_scratch.p, midx));
  }
  Prof pf(h, MG_K_VECTOR, prec);
  LK(launch_convert(MG_F64, prec, n, nrhs, e64, e, 1.0, nullptr, 0, 0.0, 0, h->st));
  return MG_OK;
}


int vcycle(mg_handle* h, int l, const void* r, void* e, int nrhs);

// e = `iters` steps of flexible GCR on A_l e = b from e = 0, preconditioned by
// the V-cycle of level l (classical Gram-Schmidt applied twice; every scalar
// stays on the device, so the whole solve is one graph-capturable sequence).
// The Krylov vectors are FP64 or FP32 (`prec`); where the level's cycle runs
// in another (16-bit) storage, each residual goes to it scaled to unit norm
// per right-hand side and the cycle's output comes back unscaled.
int coarse_gcr(mg_handle* h, int l, int prec, const void* b, void* e, int iters, int nrhs) {
  Level& a = *h->lev[l];
  const size_t n = a.n();
  const size_t vb = n * nrhs * bytes_of(prec);
  const int pl = prec_of(h, l);
  void* r = work(h, l, prec, WV_T, nrhs);
  char* W = (char*)work(h, l, prec, WV_KW, nrhs, kInnerBasis);
  char* Z = (char*)work(h, l, prec, WV_KZ, nrhs, kInnerBasis);
  void* rl = pl == prec ? nullptr : work(h, l, pl, WV_PR, nrhs);
  void* el = pl == prec ? nullptr : work(h, l, pl, WV_PE, nrhs);
  if (iters > kInnerBasis) {
    set_error("coarse_cycles above the flexible coarse solver's basis");
    return MG_EINVAL;
  }
  if (!r || !W || !Z || (pl != prec && (!rl || !el))) {
    set_error(h->capturing ? "coarse solver work buffer missing during a graph capture"
                           : "device allocation failed for the coarse solver's work vectors");
    return MG_ENOMEM;
  }
  const size_t swr = slot_inner(l), srn = swr + 4 * kMaxRhs, sbeta = srn + 4 * kMaxRhs;
  CK(cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemsetAsync(e, 0, vb, h->st));
  if (pl != prec) LK(launch_dot(prec, n, nrhs, r, r, h->red.at(srn, 4), h->st));  // ||r||^2 at srn + 2
  const double sig = sqrt((double)n) / 8.0;
  for (int k = 0; k < iters; ++k) {
    void* zk = Z + (size_t)k * vb;
    void* wk = W + (size_t)k * vb;
    if (pl == prec) {
      RET(vcycle(h, l, r, zk, nrhs));
    } else {
      LK(launch_convert(prec, pl, n, nrhs, r, rl, sig, h->red.slot(srn + 2), 4, -0.5, 0, h->st));
      RET(vcycle(h, l, rl, el, nrhs));
      LK(launch_convert(pl, prec, n, nrhs, el, zk, 1.0 / sig, h->red.slot(srn + 2), 4, 0.5, 0, h->st));
    }
    RET(op_apply(h, l, prec, zk, wk, nullptr, 1.0, 0.0, nullptr, 0, nrhs));
    Prof pf(h, MG_K_VECTOR, prec);
    if (k == 0) {
      LK(launch_dot(prec, n, nrhs, wk, r, h->red.at(swr, 4), h->st));
    } else {
      for (int pass = 0; pass < 2; ++pass) {
        LK(launch_multidot(prec, n, nrhs, k, kInnerBasis, W, n * nrhs, wk, h->red.at(sbeta, 0), h->st));
        LK(launch_multiaxpy(prec, n, nrhs, k, kInnerBasis, h->red.slot(sbeta), W, Z, n * nrhs, wk, zk, r,
                            h->red.at(swr, 4), h->st));
      }
    }
    LK(launch_gcr_update(prec, prec, n, nrhs, h->red.slot(swr), 4, wk, zk, e, r, h->red.at(srn + 2, 4), h->st));
  }
  return MG_OK;
}

// e = V_l(r): one modified V(nu_pre, nu_post) cycle on level l.
int vcycle(mg_handle* h, int l, const void* r, void* e, int nrhs) {
  const int L = (int)h->lev.size();
  const int prec = prec_of(h, l);
  if (l == L - 1) return coarsest_solve(h, l, prec, r, e, nrhs);
  Level& a = *h->lev[l];
  const int pc = prec_of(h, l + 1);
  void* res = work(h, l, prec, WV_RES, nrhs);
  void* xc = work(h, l, prec, WV_XC, nrhs);
  void* axc = work(h, l, prec, WV_AXC, nrhs);
  void* rc = work(h, l + 1, pc, WV_RC, nrhs);
  void* ec = work(h, l + 1, pc, WV_EC, nrhs);
  if (!res || !xc || !axc || !rc || !ec) {
    set_error("out of device memory for V-cycle work vectors");
    return MG_ENOMEM;
  }
  if (!a.P[prec].p) {
    set_error("prolongator of level " + std::to_string(l) + " not stored in the cycle's precision");
    return MG_EINVAL;
  }
  // pre-smoothing from e = 0
  const bool eo = l == 0 && h->p.fine_smoother == 1;
  if (eo)
    RET(eo_smooth(h, prec, r, e, false, res, h->p.nu_pre, nrhs));
  else
    RET(mr_steps(h, l, prec, r, e, true, res, h->p.nu_pre, nrhs));
  // restrict, coarse solve, prolong
  const Agg g = agg_of(a);
  const double pbytes = (double)a.Vc * 2 * a.nv * a.nhalf * a.bsites * bytes_of(prec);  // P once
  const double fbytes = (double)a.n() * bytes_of(prec) * nrhs, cbytes = (double)h->lev[l + 1]->n() * bytes_of(pc) * nrhs;
  const bool xmma = (prec == MG_F16 || prec == MG_BF16) && transfer_mma_ok(g, nrhs);
  int rvar = -1, pvar = -1;
  if (xmma) {
    DevBuf scratch;
    const size_t need = (size_t)std::max(fbytes, cbytes);
    rvar = tuned(h, tkey("restrict_mma", {prec, pc, a.nv, a.bsites, a.Vc, nrhs}), transfer_mma_variants(nrhs),
                 [&](int v) {
                   if (!scratch.p && !scratch.ensure(need)) return -1;
                   return launch_restrict(prec, prec, pc, g, a.P[prec].p, res, scratch.p, nrhs, h->st, v);
                 });
    pvar = tuned(h, tkey("prolong_mma", {prec, pc, a.nv, a.bsites, a.Vc, nrhs}), transfer_mma_variants(nrhs),
                 [&](int v) {
                   if (!scratch.p && !scratch.ensure(need)) return -1;
                   return launch_prolong(pc, prec, prec, g, a.P[prec].p, rc, scratch.p, nrhs, h->st, v);
                 });
  }
  {
    Prof pf(h, MG_K_RESTRICT, prec, pbytes + fbytes + cbytes);
    LK(launch_restrict(prec, prec, pc, g, a.P[prec].p, res, rc, nrhs, h->st, rvar));
  }
  if (l + 1 == L - 1) {
    RET(coarsest_solve(h, l + 1, pc, rc, ec, nrhs));
  } else {
    if (h->p.coarse_solver == 0 && (pc == MG_F64 || pc == MG_F32)) {
      RET(coarse_gcr(h, l + 1, pc, rc, ec, a.cycles, nrhs));
    } else {
      RET(vcycle(h, l + 1, rc, ec, nrhs));
      void* t = work(h, l + 1, pc, WV_T, nrhs);
      void* dt = work(h, l + 1, pc, WV_DT, nrhs);
      if (!t || !dt) return MG_ENOMEM;
      for (int c = 1; c < a.cycles; ++c) {
        RET(op_apply(h, l + 1, pc, ec, t, rc, -1.0, 1.0, nullptr, 0, nrhs));
        RET(vcycle(h, l + 1, t, dt, nrhs));
        Prof pf(h, MG_K_VECTOR, pc);
        LK(launch_convert(pc, pc, h->lev[l + 1]->n(), nrhs, dt, ec, 1.0, nullptr, 0, 0.0, 1, h->st));
      }
    }
  }
  {
    Prof pf(h, MG_K_PROLONG, prec, pbytes + fbytes + cbytes);
    LK(launch_prolong(pc, prec, prec, g, a.P[prec].p, ec, xc, nrhs, h->st, pvar));
  }
  // alpha = <A x_c|r0> / <A x_c|A x_c>  (Eq. 3.5);  e += alpha x_c, r0 -= alpha A x_c
  const size_t sl = slot_level(l);
  RET(op_apply(h, l, prec, xc, axc, nullptr, 1.0, 0.0, res, sl, nrhs));
  RET(mr_update(h, l, prec, e, e, xc, res, res, axc, sl, 1.0, nrhs));
  // post-smoothing
  if (eo) return eo_smooth(h, prec, res, e, true, res, h->p.nu_post, nrhs);
  RET(mr_steps(h, l, prec, res, e, false, res, h->p.nu_post, nrhs));
  return MG_OK;
}

// e = V_0(r) through a CUDA graph of the whole cycle.  The first call for a
// given (nrhs, r, e) runs the cycle eagerly (so every work buffer exists),
// then captures it on a private stream; later calls replay the graph on the
// handle's stream.  Any buffer reallocation invalidates the cached graphs.
int vcycle_graph(mg_handle* h, const void* r, void* e, int nrhs) {
  if (!h->use_graphs || h->prof_mask) return vcycle(h, 0, r, e, nrhs);  // the profiler times launches one by one
  for (auto& g : h->graphs) {
    if (g.mm == h->mm_active && g.nrhs == nrhs && g.in == r && g.out == e && g.gen == h->buf_gen) {
      CK(cudaGraphLaunch(g.exec, h->st));
      count_launches(g.nodes);
      return MG_OK;
    }
  }
  RET(vcycle(h, 0, r, e, nrhs));  // eager run: allocates and warms every buffer
  if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
  CK(cudaStreamSynchronize(h->st));
  cudaStream_t keep = h->st;
  const unsigned long long gen = h->buf_gen;
  const unsigned long long n0 = tl_launches;  // this thread's: other threads launch meanwhile
  h->st = h->cap_st;
  h->capturing = true;
  cudaGraph_t graph = nullptr;
  int rc = MG_OK;
  cudaError_t ce;
  {
    // no device-wide synchronisation (which would invalidate the capture) while it runs
    std::shared_lock<std::shared_mutex> nosync(g_capture_mu);
    ce = cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      rc = vcycle(h, 0, r, e, nrhs);
      ce = cudaStreamEndCapture(h->cap_st, &graph);
    }
  }
  h->capturing = false;
  h->st = keep;
  const unsigned long long nodes = tl_launches - n0;
  // a capture launches nothing: its kernels count when the graph is replayed
  __atomic_fetch_sub(&g_launches, nodes, __ATOMIC_RELAXED);
  tl_launches = n0;
  if (ce != cudaSuccess || rc != MG_OK || gen != h->buf_gen) {
    // the eager run above already produced e; a capture that failed only costs the graph
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    take_launch_error();
    h->use_graphs = false;  // fall back to eager launches for this handle
    return MG_OK;
  }
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    h->use_graphs = false;
    return MG_OK;
  }
  // drop graphs of older generations
  for (auto it = h->graphs.begin(); it != h->graphs.end();) {
    if (it->gen != h->buf_gen) {
      cudaGraphExecDestroy(it->exec);
      it = h->graphs.erase(it);
    } else {
      ++it;
    }
  }
  h->graphs.push_back({h->mm_active, nrhs, r, e, gen, nodes, exec});
  return MG_OK;
}

// Pinned host mirrors of the reduction slots, reused across handles (freeing
// pinned memory synchronises the device, which a graph capture on another
// thread must not see).
std::mutex g_host_slots_mu;
std::vector<double*> g_host_slots;
double* take_host_slots() {
  {
    std::lock_guard<std::mutex> lk(g_host_slots_mu);
    if (!g_host_slots.empty()) {
      double* p = g_host_slots.back();
      g_host_slots.pop_back();
      return p;
    }
  }
  double* p = nullptr;
  if (cudaMallocHost((void**)&p, slot_total() * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void give_host_slots(double* p) {
  std::lock_guard<std::mutex> lk(g_host_slots_mu);
  g_host_slots.push_back(p);
}

int read_slots(mg_handle* h, size_t off, int count) {
  CK(cudaMemcpyAsync(h->host_slots, h->red.slot(off), count * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return MG_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

const char* mg_last_error(void) { return g_err.c_str(); }

int mg_default_params(mg_params* p) {
  if (!p) return MG_EINVAL;
  memset(p, 0, sizeof(*p));
  p->n_levels = 2;
  for (int l = 0; l < MG_MAX_LEVELS - 1; ++l) {
    for (int m = 0; m < 4; ++m) p->block[l][m] = 4;
    p->nv[l] = 20;
    p->setup_sweeps[l] = 20;
    p->coarse_cycles[l] = 1;
  }
  p->coarse_cycles[0] = 4;
  p->nu_pre = 2;
  p->nu_post = 2;
  p->omega = 0.8;
  p->gcr_restart = 50;
  p->max_iter = 2000;
  p->mixed = 0;
  p->fine_prec = MG_F16;
  p->coarse_prec = MG_F32;
  p->reliable_delta = 1e-4;
  p->seed = 0;
  p->use_graphs = 1;
  p->adapt_cycles = 16;
  return MG_OK;
}

int mg_destroy(mg_handle* h) {
  if (!h) return MG_OK;
  // the handle's buffers may have served any stream a caller passed: wait for all of them once,
  // then return the buffers to the cache without a synchronisation each (if the synchronisation
  // fails, every buffer takes the cautious path of DevBuf::release)
  bool synced = false;
  {
    std::unique_lock<std::shared_mutex> nocapture(g_capture_mu, std::try_to_lock);
    if (nocapture.owns_lock()) synced = cudaDeviceSynchronize() == cudaSuccess;
  }
  if (!synced) {
    cudaGetLastError();
    if (h->st) cudaStreamSynchronize(h->st);  // at least the handle's own stream; buffers take the cautious path
  }
  if (h->host_slots) give_host_slots(h->host_slots);
  for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  if (synced) {
    DevIdleScope idle;
    delete h;
  } else {
    delete h;
  }
  cudaGetLastError();
  return MG_OK;
}

size_t mg_trim_cache(void) { return wmg::dev_cache().trim(); }

size_t mg_release_work(mg_handle* h, void* stream) {
  if (!h) return 0;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess || cudaStreamSynchronize(h->st) != cudaSuccess) {
    cudaGetLastError();
    return 0;  // work may still be queued on the buffers: keep them
  }
  DevIdleScope idle;  // both streams the handle's solves use are done
  size_t freed = 0;
  auto drop = [&](DevBuf& d) {
    if (d.p) {
      freed += d.bytes;
      d.release();
    }
  };
  for (auto& byprec : h->work)
    for (auto& vecs : byprec)
      for (auto& v : vecs)
        if (v) drop(*v);
  for (DevBuf* d : {&h->gr, &h->gW, &h->gZ, &h->gb64, &h->gx64, &h->gr64, &h->gtmp, &h->gH, &h->galpha, &h->gy,
                    &h->mm_inv})
    drop(*d);
  h->mm_masses.clear();
  ++h->buf_gen;  // captured cycles hold the released addresses
  return freed;
}

size_t mg_handle_bytes(const mg_handle* h) {
  if (!h) return 0;
  size_t b = 0;
  auto add = [&](const DevBuf& d) { b += d.p ? d.bytes : 0; };
  for (const auto& lp : h->lev) {
    const Level& a = *lp;
    for (int q = 0; q < 4; ++q) {
      add(a.links[q]);
      add(a.links_eo[q]);
      add(a.cop[q]);
      add(a.P[q]);
    }
    add(a.cop_mma);
    add(a.inv);
    add(a.mm_scratch);
  }
  for (const auto& byprec : h->work)
    for (const auto& vecs : byprec)
      for (const auto& v : vecs)
        if (v) add(*v);
  add(h->red.partials);
  add(h->red.tickets);
  add(h->red.slots);
  for (const DevBuf* d : {&h->gr, &h->gW, &h->gZ, &h->gb64, &h->gx64, &h->gr64, &h->gtmp, &h->gH, &h->galpha, &h->gy,
                          &h->err_flag, &h->mm_adiag, &h->mm_shift, &h->mm_idx, &h->mm_inv})
    add(*d);
  return b;
}

// Dense inverse of the coarsest level (FP64, or FP32 refined in FP64 in the mixed form).
// Dense inverse of the coarsest operator of each handle (Sec. 4: exact
// coarsest solve), FP64 (plain) or FP32 (mixed).  Handles of one batch share
// the coarsest geometry (retargets of one hierarchy) and every elimination
// launch.
static int build_coarsest_many(mg_handle* const* hs, int count) {
  mg_handle* h0 = hs[0];
  const int Lv = (int)h0->lev.size();
  if (Lv < 2) return MG_OK;
  cudaStream_t st = h0->st;
  const Level& c0 = *h0->lev[Lv - 1];
  const size_t N = c0.n();
  if (N > 8192) {
    set_error("coarsest level has " + std::to_string(N) + " unknowns; the dense solve takes at most 8192");
    return MG_EINVAL;
  }
  const int prec = (h0->p.mixed && !h0->p.coarsest_f64) ? MG_F32 : MG_F64;
  const size_t eb = bytes_of(prec);
  DevBuf aug, col, errflag, blk;
  const size_t bb = gjb_scratch_bytes((int)N, eb, count);
  if (!aug.ensure(N * 2 * N * eb * count) || !col.ensure(dense_inverse_scratch_bytes(prec, (int)N) * count) ||
      !errflag.ensure(sizeof(int) * count) || (bb && !blk.ensure(bb)))
    return MG_ENOMEM;
  std::vector<const double2*> C(count);
  std::vector<void*> inv(count);
  for (int z = 0; z < count; ++z) {
    Level& c = *hs[z]->lev[Lv - 1];
    c.inv_prec = prec;
    if (!c.inv.ensure(N * N * eb) || !c.mm_scratch.ensure(dense_matvec_scratch_bytes((int)N))) return MG_ENOMEM;
    // the product's tickets sit after the partial tiles, at an offset that depends on N
    CK(cudaMemsetAsync(c.mm_scratch.p, 0, dense_matvec_scratch_bytes((int)N), st));
    C[z] = c.cop[MG_F64].as<double2>();
    inv[z] = c.inv.p;
  }
  CK(cudaMemsetAsync(errflag.p, 0, sizeof(int) * count, st));
  long long nl = 1;
  {
    Prof pf(h0, MG_K_INVERSE, prec);
    LK(dense_inverse_batch(prec, C.data(), c0.L, c0.ncomp, count, aug.p, col.p, errflag.as<int>(), inv.data(),
                           blk.p, st, &nl));
  }
  count_launches(nl - 1);
  std::vector<int> herr(count, 0);
  CK(cudaMemcpyAsync(herr.data(), errflag.p, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (DevBuf* t : {&aug, &col, &errflag, &blk}) t->release_idle();  // their only stream is done
  for (int z = 0; z < count; ++z)
    if (herr[z]) {
      set_error("coarsest operator is singular (zero pivot)");
      return MG_EINVAL;
    }
  return MG_OK;
}

static int build_coarsest(mg_handle* h) {
  RET(build_coarsest_many(&h, 1));
  if (h->lev.size() >= 2) h->lev.back()->inv_pending = false;
  return MG_OK;
}

// Inverses of the coarsest operator at each of `ms` (the level's FP64 stencil
// shifted by m - mass on the diagonal, as mg_retarget does), built together
// into h->mm_inv = [count][N][N] for solves with a mass per right-hand side.
static int build_mass_inverses(mg_handle* h, const std::vector<double>& ms) {
  cudaStream_t st = h->st;
  Level& c = *h->lev.back();
  const size_t N = c.n();
  if (N > 8192) {
    set_error("coarsest level has " + std::to_string(N) + " unknowns; the dense solve takes at most 8192");
    return MG_EINVAL;
  }
  const int count = (int)ms.size();
  const int prec = (h->p.mixed && !h->p.coarsest_f64) ? MG_F32 : MG_F64;
  const size_t eb = bytes_of(prec), cb = (size_t)9 * c.ncomp * c.ncomp * c.V * 16;
  DevBuf shifted, aug, col, errflag, blk;
  const size_t bb = gjb_scratch_bytes((int)N, eb, count);
  const void* before = h->mm_inv.p;
  if (!shifted.ensure(cb * count) || !aug.ensure(N * 2 * N * eb * count) ||
      !col.ensure(dense_inverse_scratch_bytes(prec, (int)N) * count) || !errflag.ensure(sizeof(int) * count) ||
      (bb && !blk.ensure(bb)) || !h->mm_inv.ensure(N * N * eb * count))
    return MG_ENOMEM;
  if (h->mm_inv.p != before) ++h->buf_gen;  // captured cycles hold the old address
  std::vector<const double2*> C(count);
  std::vector<void*> inv(count);
  for (int z = 0; z < count; ++z) {
    char* sz = (char*)shifted.p + cb * z;
    CK(cudaMemcpyAsync(sz, c.cop[MG_F64].p, cb, cudaMemcpyDeviceToDevice, st));
    if (ms[z] != h->mass) LK(launch_diag_shift((double2*)sz, c.ncomp, c.V, ms[z] - h->mass, st));
    C[z] = (const double2*)sz;
    inv[z] = (char*)h->mm_inv.p + N * N * eb * z;
  }
  CK(cudaMemsetAsync(errflag.p, 0, sizeof(int) * count, st));
  long long nl = 1;
  {
    Prof pf(h, MG_K_INVERSE, prec);
    LK(dense_inverse_batch(prec, C.data(), c.L, c.ncomp, count, aug.p, col.p, errflag.as<int>(), inv.data(), blk.p,
                           st, &nl));
  }
  count_launches(nl - 1);
  std::vector<int> herr(count, 0);
  CK(cudaMemcpyAsync(herr.data(), errflag.p, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (DevBuf* t : {&shifted, &aug, &col, &errflag, &blk}) t->release_idle();  // their only stream is done
  for (int z = 0; z < count; ++z)
    if (herr[z]) {
      set_error("coarsest operator is singular (zero pivot) at one of the masses");
      return MG_EINVAL;
    }
  c.inv_prec = prec;
  h->mm_masses = ms;
  return MG_OK;
}

// A deferred coarsest inverse is built before the first cycle that needs it.
static int ensure_coarsest(mg_handle* h) {
  if (h->lev.size() >= 2 && h->lev.back()->inv_pending) RET(build_coarsest(h));
  return MG_OK;
}

// ------------------------------------------------------------------ setup pieces
// Geometry of the aggregation of level l into level l+1.
static int init_level(mg_handle* h, int l) {
  const mg_params& p = h->p;
  Level& a = *h->lev[l];
  a.nv = p.nv[l];
  a.sweeps = p.setup_sweeps[l];
  a.cycles = p.coarse_cycles[l] < 1 ? 1 : p.coarse_cycles[l];
  a.nhalf = a.ncomp / 2;
  a.bsites = 1;
  a.Vc = 1;
  for (int m = 0; m < 4; ++m) {
    a.blk[m] = p.block[l][m];
    if (a.blk[m] < 1 || a.L[m] % a.blk[m]) {
      set_error("level " + std::to_string(l) + ": extent not divisible by the block size");
      return MG_EINVAL;
    }
    a.Lc[m] = a.L[m] / a.blk[m];
    a.bsites *= a.blk[m];
    a.Vc *= a.Lc[m];
  }
  if (a.nv < 1 || a.nv > a.nhalf * a.bsites) {
    set_error("level " + std::to_string(l) + ": nv must be in [1, ncomp/2 * block sites]");
    return MG_EINVAL;
  }
  // The Galerkin product holds one block of a P column in shared memory.
  const size_t gal = galerkin_smem_bytes(p.mixed ? MG_F32 : MG_F64, a.ncomp, a.bsites, a.nv);
  if (gal > kGalerkinSmemMax) {
    set_error("level " + std::to_string(l) + ": a block of " + std::to_string(a.bsites) + " sites x " +
              std::to_string(a.ncomp) + " components needs " + std::to_string(gal) +
              " B of shared memory in the Galerkin product (at most " + std::to_string(kGalerkinSmemMax) +
              "); use smaller blocks");
    return MG_EINVAL;
  }
  return ensure_reducer(h, a.nv);
}

// The Nv random start vectors of level l, FP64 [nv][ncomp][V]: the caller's
// (host, external layout) or the counter-based Gaussian generator's.  Both
// are defined on the final hierarchy, where level l >= 1 has 2 nv[l-1]
// components; while the level above still has k < nv[l-1] candidates, the
// starts are restricted to the first k components of each chirality half.
static int make_starts(mg_handle* h, int l, const double* start, DevBuf& S) {
  cudaStream_t st = h->st;
  Level& a = *h->lev[l];
  const int nfull = l == 0 ? 12 : 2 * h->p.nv[l - 1];
  const size_t vbf = (size_t)nfull * a.V * 16, vb = a.n() * 16;
  DevBuf full;
  if (!full.ensure(vbf * a.nv) || !S.ensure(vb * a.nv)) return MG_ENOMEM;
  if (start) {
    DevBuf ext;
    if (!ext.ensure(vbf * a.nv)) return MG_ENOMEM;
    CK(cudaMemcpyAsync(ext.p, start, vbf * a.nv, cudaMemcpyHostToDevice, st));
    LK(launch_ext_to_int(MG_F64, nfull, a.q, a.V, a.nv, ext.p, full.p, st));
  } else {
    Prof pf(h, MG_K_SETUP, MG_F64);
    LK(launch_gaussian_starts(h->p.seed + (uint64_t)l, a.nv, nfull, a.q, a.V, full.p, st));
  }
  if (nfull == a.ncomp) {
    CK(cudaMemcpyAsync(S.p, full.p, vb * a.nv, cudaMemcpyDeviceToDevice, st));
  } else {
    const size_t half = (size_t)(a.ncomp / 2) * a.V * 16, fhalf = (size_t)(nfull / 2) * a.V * 16;
    CK(cudaMemcpy2DAsync(S.p, vb, full.p, vbf, half, a.nv, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpy2DAsync((char*)S.p + half, vb, (char*)full.p + fhalf, vbf, half, a.nv, cudaMemcpyDeviceToDevice,
                         st));
  }
  CK(cudaStreamSynchronize(st));
  return MG_OK;
}

// Sec. 2 adaptive steps 1-2: `sweeps` MR steps on A x = 0 from the k FP64
// vectors at x64 (all of them right-hand sides of one launch), then unit
// normalisation, in place.
static int relax_candidates(mg_handle* h, int l, void* x64, int k) {
  const mg_params& p = h->p;
  cudaStream_t st = h->st;
  Level& a = *h->lev[l];
  const int rp = p.mixed ? MG_F32 : MG_F64;  // the mixed form relaxes in FP32
  DevBuf candr, rr, pp, rr2, pp2;
  void* x = x64;
  const size_t vr = a.n() * bytes_of(rp);
  if (rp != MG_F64) {
    if (!candr.ensure(vr * k)) return MG_ENOMEM;
    LK(launch_convert(MG_F64, rp, a.n(), k, x64, candr.p, 1.0, nullptr, 0, 0.0, 0, st));
    x = candr.p;
  }
  // level 0 on small lattices: each step's update is fused into the next step's stencil (r and p
  // ping-pong).  The fused stencil reads r and p at all nine points; once the candidates no longer fit
  // in L2 that costs more than the separate update pass it saves.
  const bool fuse = l == 0 && (size_t)a.V * k <= kFuseRelaxSites;
  if (!rr.ensure(vr * k) || !pp.ensure(vr * k) || (fuse && (!rr2.ensure(vr * k) || !pp2.ensure(vr * k))))
    return MG_ENOMEM;
  RET(ensure_reducer(h, k));
  const size_t sl = slot_level(l);
  if (a.sweeps > 0) {
    void *r = rr.p, *pv = pp.p, *r2 = rr2.p, *p2 = pp2.p;
    RET(op_apply(h, l, rp, x, r, nullptr, -1.0, 0.0, nullptr, 0, k));
    bool owed = false;  // the update of (x, r) with the last p and its dots is still to be applied
    for (int s = 0; s < a.sweeps; ++s) {
      // FP32 relaxation: the recursively updated residual drifts from -A x
      // once it has shrunk by a few orders, so it is recomputed every
      // kTrueResidualEvery steps (FP64 follows the plain recursion).
      const bool recompute = rp != MG_F64 && s > 0 && s % kTrueResidualEvery == 0;
      if (owed && (!fuse || recompute)) {
        RET(mr_update(h, l, rp, x, x, r, r, r, pv, sl, p.omega, k));
        owed = false;
      }
      if (recompute) RET(op_apply(h, l, rp, x, r, nullptr, -1.0, 0.0, nullptr, 0, k));
      if (owed) {  // x += c r, r' = r - c p, p' = A r' and its dots, in one launch
        RET(mr_fused(h, rp, r, pv, nullptr, x, x, r2, p2, sl, p.omega, k));
        std::swap(r, r2);
        std::swap(pv, p2);
      } else {
        RET(op_apply(h, l, rp, r, pv, nullptr, 1.0, 0.0, r, sl, k));
      }
      owed = true;
    }
    RET(mr_update(h, l, rp, x, x, r, r, r, pv, sl, p.omega, k));
  }
  LK(launch_dot(rp, a.n(), k, x, x, h->red.at(slot_misc(), 4), st));
  LK(launch_convert(rp, MG_F64, a.n(), k, x, x64, 1.0, h->red.slot(slot_misc() + 2), 4, -0.5, 0, st));
  CK(cudaStreamSynchronize(st));
  return MG_OK;
}

// A_{l+1} = P_l^+ A_l P_l (Sec. 2) from the current P_l and A_l: FP64
// arithmetic for the plain hierarchy, FP32 for the mixed one, stored in FP64;
// then the precision copies of A_{l+1} the cycle and the relaxation use.
static int galerkin(mg_handle* h, int l) {
  const mg_params& p = h->p;
  cudaStream_t st = h->st;
  const int Lv = p.n_levels;
  Level& a = *h->lev[l];
  Level& c = *h->lev[l + 1];
  const int nc = c.ncomp;
  const Agg g = agg_of(a);
  if (!c.cop[MG_F64].ensure((size_t)9 * nc * nc * c.V * 16)) return MG_ENOMEM;
  const int gp = p.mixed ? MG_F32 : MG_F64;
  const size_t vbg = a.n() * bytes_of(gp);
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(nc, ((size_t)1 << 30) / vbg));
  DevBuf cols;
  if (!cols.ensure(vbg * chunk)) return MG_ENOMEM;
  for (int j0 = 0; j0 < nc; j0 += chunk) {
    const int ncols = std::min(chunk, nc - j0);
    {
      Prof pf(h, MG_K_SETUP, gp);
      LK(launch_p_column(gp, g, a.P[gp].p, j0, ncols, cols.p, st));
    }
    Prof pf(h, MG_K_GALERKIN, gp);
    if (l == 0)
      LK(launch_galerkin_wilson(gp, g, a.links[gp].p, h->mass, cols.p, a.P[gp].p, j0, ncols,
                                c.cop[MG_F64].as<double2>(), st));
    else
      LK(launch_galerkin_stencil(gp, g, a.cop[gp].p, cols.p, a.P[gp].p, j0, ncols, c.cop[MG_F64].as<double2>(),
                                 st));
  }
  if (p.mixed && l + 2 < Lv) {
    const size_t ncop = (size_t)9 * nc * nc * c.V;
    const int want[2] = {MG_F32, p.coarse_prec};
    for (int q : want) {
      if (!c.cop[q].ensure(ncop * bytes_of(q))) return MG_ENOMEM;
      LK(launch_convert(MG_F64, q, ncop, 1, c.cop[MG_F64].p, c.cop[q].p, 1.0, nullptr, 0, 0.0, 0, st));
    }
    if (p.coarse_mma) {
      if (!c.cop_mma.ensure(mma_pack_bytes(nc, c.V))) return MG_ENOMEM;
      LK(launch_mma_pack(c.cop[MG_F64].as<double2>(), nc, c.V, c.cop_mma.p, st));
    }
  }
  return MG_OK;
}

// P_l from FP64 candidates (Sec. 2 step 3, Eq. 2.3: blockwise Gram-Schmidt,
// chirality kept), its precision copies, then A_{l+1} (level l+1 is created
// on first use).
static int build_level(mg_handle* h, int l, DevBuf& cand) {
  const mg_params& p = h->p;
  cudaStream_t st = h->st;
  Level& a = *h->lev[l];
  const Agg g = agg_of(a);
  const size_t np = (size_t)a.Vc * 2 * a.nv * a.nhalf * a.bsites;
  DevBuf errflag;
  if (!errflag.ensure(sizeof(int)) || !a.P[MG_F64].ensure(np * 16)) return MG_ENOMEM;
  CK(cudaMemsetAsync(errflag.p, 0, sizeof(int), st));
  {
    Prof pf(h, MG_K_SETUP, MG_F64);
    LK(launch_block_gs(g, cand.as<double2>(), a.P[MG_F64].as<double2>(), errflag.as<int>(), st));
  }
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, errflag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr == 2) {
    set_error("block Gram-Schmidt lost rank on level " + std::to_string(l));
    return MG_ERANK;
  }
  const int copies[2] = {p.mixed ? MG_F32 : MG_F64, prec_of(h, l)};
  for (int pr : copies) {
    if (pr == MG_F64) continue;
    if (!a.P[pr].ensure(np * bytes_of(pr))) return MG_ENOMEM;
    LK(launch_convert(MG_F64, pr, np, 1, a.P[MG_F64].p, a.P[pr].p, 1.0, nullptr, 0, 0.0, 0, st));
  }
  if ((int)h->lev.size() == l + 1) h->lev.emplace_back(new Level());
  Level& c = *h->lev[l + 1];  // its size follows the current number of candidates
  for (int m = 0; m < 4; ++m) c.L[m] = a.Lc[m];
  c.V = a.Vc;
  c.ncomp = 2 * a.nv;
  return galerkin(h, l);
}

// One adaptive step of Sec. 2 for the q FP64 vectors at x64 (random starts):
// `iters` iterations of the current solver -- flexible GCR preconditioned by
// the multigrid cycle of level l, restarted every kInnerBasis iterations --
// on A x = 0 from x, all q as right-hand sides of one batched solve, then unit
// normalisation, in place.  x stays FP64; each restart solves A e = -A x with
// FP64 or FP32 Krylov vectors (the mixed form) from the residual scaled to
// unit norm per right-hand side, and adds e to x.
static int adapt_candidates(mg_handle* h, int l, void* x64, int q, int iters) {
  cudaStream_t st = h->st;
  Level& a = *h->lev[l];
  const size_t n = a.n();
  const int pg = prec_of(h, l) == MG_F64 ? MG_F64 : MG_F32;
  DevBuf R, Rg, Eg;
  if (!R.ensure(n * 16 * q) || !Rg.ensure(n * bytes_of(pg) * q) || !Eg.ensure(n * bytes_of(pg) * q))
    return MG_ENOMEM;
  RET(ensure_reducer(h, q));
  const double sig = sqrt((double)n) / 8.0;
  for (int done = 0; done < iters; done += kInnerBasis) {
    const int k = std::min(kInnerBasis, iters - done);
    RET(op_apply(h, l, MG_F64, x64, R.p, nullptr, -1.0, 0.0, nullptr, 0, q));
    LK(launch_dot(MG_F64, n, q, R.p, R.p, h->red.at(slot_misc(), 4), st));
    LK(launch_convert(MG_F64, pg, n, q, R.p, Rg.p, sig, h->red.slot(slot_misc() + 2), 4, -0.5, 0, st));
    RET(coarse_gcr(h, l, pg, Rg.p, Eg.p, k, q));
    LK(launch_convert(pg, MG_F64, n, q, Eg.p, x64, 1.0 / sig, h->red.slot(slot_misc() + 2), 4, 0.5, 1, st));
  }
  LK(launch_dot(MG_F64, n, q, x64, x64, h->red.at(slot_misc(), 4), st));
  LK(launch_convert(MG_F64, MG_F64, n, q, x64, x64, 1.0, h->red.slot(slot_misc() + 2), 4, -0.5, 0, st));
  CK(cudaStreamSynchronize(st));
  return MG_OK;
}

// Levels l .. coarsest from the operator of level l (Sec. 2): V^k of level l
// starts as the first Nv - adapt_nv[l] relaxed candidates; each of the
// adapt_steps adaptive steps appends a batch of candidates made by the
// current solver (whose cycle needs the levels below, rebuilt by the same
// procedure after every change of P_l).  Batch s holds
// adapt_nv / steps candidates, one more for s < adapt_nv % steps.
static int build_from(mg_handle* h, int l, const double* const* starts) {
  const mg_params& p = h->p;
  if (l + 1 >= p.n_levels) {
    // deferred: only without adaptive steps, whose cycles need the coarsest solve during setup
    if (p.defer_coarsest && p.adapt_steps == 0 && l > 0) {
      h->lev[l]->inv_pending = true;
      return MG_OK;
    }
    return build_coarsest(h);
  }
  RET(init_level(h, l));
  Level& a = *h->lev[l];
  const int nv = a.nv;
  int na = p.adapt_steps > 0 ? p.adapt_nv[l] : 0;
  if (na < 0 || na >= nv) {
    set_error("level " + std::to_string(l) + ": adapt_nv must be in [0, nv)");
    return MG_EINVAL;
  }
  const int steps = std::min(p.adapt_steps, na);
  const int k0 = nv - na;
  const size_t vb = a.n() * 16;
  DevBuf cand;
  RET(make_starts(h, l, starts ? starts[l] : nullptr, cand));
  RET(relax_candidates(h, l, cand.p, k0));
  a.nv = k0;
  RET(build_level(h, l, cand));
  RET(build_from(h, l + 1, starts));
  for (int s = 0; s < steps; ++s) {
    const int q = na / steps + (s < na % steps ? 1 : 0);
    Level& al = *h->lev[l];
    RET(adapt_candidates(h, l, (char*)cand.p + vb * al.nv, q, p.adapt_cycles < 1 ? 1 : p.adapt_cycles));
    al.nv += q;
    RET(build_level(h, l, cand));
    RET(build_from(h, l + 1, starts));
  }
  return MG_OK;
}

// Largest deviation of an input link from SU(3) that mg_setup accepts.
const double kSu3Tolerance = 1e-10;

static int setup_impl(mg_handle* h, const double* gauge, int gauge_on_device, const double* const* starts) {
  const mg_params& p = h->p;
  cudaStream_t st = h->st;
  // ---- level 0 and the gauge field
  h->lev.emplace_back(new Level());
  Level& f = *h->lev[0];
  for (int m = 0; m < 4; ++m) f.L[m] = h->dims[m];
  f.V = f.L[0] * f.L[1] * f.L[2] * f.L[3];
  f.ncomp = 12;
  f.q = 4;
  {
    DevBuf ext;
    const double* gdev = gauge;
    const size_t gbytes = (size_t)4 * f.V * 9 * 16;
    if (!gauge_on_device) {
      if (!ext.ensure(gbytes)) return MG_ENOMEM;
      CK(cudaMemcpyAsync(ext.p, gauge, gbytes, cudaMemcpyHostToDevice, st));
      gdev = ext.as<double>();
    }
    // the 12-real link storage of the FP32 / 16-bit operators rebuilds the third row as for SU(3)
    {
      DevBuf chk;
      if (!chk.ensure(sizeof(unsigned))) return MG_ENOMEM;
      CK(cudaMemsetAsync(chk.p, 0, sizeof(unsigned), st));
      LK(launch_su3_check(gdev, f.V, chk.as<unsigned>(), st));
      unsigned bits = 0u;
      CK(cudaMemcpyAsync(&bits, chk.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      float dev = 0.f;
      memcpy(&dev, &bits, sizeof(dev));
      if (!(dev <= kSu3Tolerance)) {
        char msg[160];
        snprintf(msg, sizeof msg, "gauge field is not SU(3): max |U U^+ - 1|, |det U - 1| over the links = %.3g",
                 (double)dev);
        set_error(msg);
        return MG_EINVAL;
      }
    }
    std::vector<int> precs = {MG_F64};
    if (p.mixed) {
      precs.push_back(MG_F32);
      if (p.fine_prec != MG_F32 && p.fine_prec != MG_F64) precs.push_back(p.fine_prec);
    }
    for (int pr : precs) {
      const int NL = pr == MG_F64 ? 9 : 6;
      if (!f.links[pr].ensure((size_t)4 * NL * f.V * bytes_of(pr))) return MG_ENOMEM;
      LK(launch_pack_links(pr, gdev, f.links[pr].p, f.V, st));
    }
    CK(cudaStreamSynchronize(st));
  }
  RET(ensure_reducer(h, 1));
  // ---- coarser levels (Sec. 2): candidates, P, the Galerkin operators, the
  // coarsest inverse
  RET(build_from(h, 0, starts));
  CK(cudaStreamSynchronize(st));
  return MG_OK;
}

int mg_setup(mg_handle** hout, const double* gauge, int gauge_on_device, const int dims[4], double mass,
             const mg_params* p, const double* const* starts, void* stream) {
  if (!hout) return MG_EINVAL;
  *hout = nullptr;
  if (!gauge || !dims || !p) {
    set_error("null argument");
    return MG_EINVAL;
  }
  for (int m = 0; m < 4; ++m)
    if (dims[m] < 1) {
      set_error("dims must be >= 1");
      return MG_EINVAL;
    }
  if ((double)dims[0] * dims[1] * dims[2] * dims[3] > (double)kMaxSites) {
    set_error("lattice above 2^26 sites (the level-0 kernels index one field in 32 bits)");
    return MG_EINVAL;
  }
  if (p->n_levels < 1 || p->n_levels > MG_MAX_LEVELS || p->nu_pre < 0 || p->nu_post < 0 || p->gcr_restart < 1 ||
      p->gcr_restart > kMaxBasis || !(p->omega > 0.0)) {
    set_error("invalid mg_params (levels 1..4, restart 1..64, nu >= 0, omega > 0)");
    return MG_EINVAL;
  }
  if (p->mixed && (check_prec(p->fine_prec) || p->fine_prec == MG_F64 || check_prec(p->coarse_prec) ||
                   p->coarse_prec == MG_F64)) {
    set_error("mixed precision needs fine_prec and coarse_prec in {F32, F16, BF16}");
    return MG_EINVAL;
  }
  if (p->mixed && p->coarse_prec != MG_F32 && p->coarse_prec != p->fine_prec) {
    set_error("mixed precision needs coarse_prec == F32 or coarse_prec == fine_prec (the transfer kernels' pairs)");
    return MG_EINVAL;
  }
  if (p->fine_smoother != 0 && p->fine_smoother != 1) {
    set_error("fine_smoother must be 0 (MR) or 1 (even-odd)");
    return MG_EINVAL;
  }
  for (int l = 0; l + 2 < p->n_levels; ++l)
    if (p->coarse_solver == 0 && p->coarse_cycles[l] > kInnerBasis) {
      set_error("coarse_cycles above " + std::to_string(kInnerBasis) +
                " (the flexible coarse solver keeps that many directions)");
      return MG_EINVAL;
    }
  if (p->fine_smoother == 1 && (dims[0] % 2 || dims[1] % 2 || dims[2] % 2 || dims[3] % 2)) {
    set_error("the even-odd smoother needs every lattice extent even");
    return MG_EINVAL;
  }
  mg_handle* h = new mg_handle();
  h->p = *p;
  h->mass = mass;
  for (int m = 0; m < 4; ++m) h->dims[m] = dims[m];
  h->st = (cudaStream_t)stream;
  h->use_graphs = p->use_graphs != 0;
  h->prof_mask = __atomic_load_n(&g_default_prof_mask, __ATOMIC_RELAXED);
  if ((h->host_slots = take_host_slots()) == nullptr) {
    cudaGetLastError();
    delete h;
    set_error("pinned host allocation failed");
    return MG_ENOMEM;
  }
  int rc = setup_impl(h, gauge, gauge_on_device, starts);
  if (rc != MG_OK) {
    mg_destroy(h);
    return rc;
  }
  *hout = h;
  return MG_OK;
}

static int retarget_impl(const mg_handle* src, mg_handle* h, bool coarsest = true) {
  cudaStream_t st = h->st;
  const double delta = h->mass - src->mass;
  for (size_t l = 0; l < src->lev.size(); ++l) {
    const Level& a = *src->lev[l];
    h->lev.emplace_back(new Level());
    Level& b = *h->lev[l];
    for (int m = 0; m < 4; ++m) {
      b.L[m] = a.L[m];
      b.blk[m] = a.blk[m];
      b.Lc[m] = a.Lc[m];
    }
    b.V = a.V;
    b.ncomp = a.ncomp;
    b.q = a.q;
    b.nv = a.nv;
    b.bsites = a.bsites;
    b.nhalf = a.nhalf;
    b.Vc = a.Vc;
    b.sweeps = a.sweeps;
    b.cycles = a.cycles;
    for (int pr = 0; pr < 4; ++pr) {
      const DevBuf* from[4] = {&a.links[pr], &a.cop[pr], &a.P[pr], &a.links_eo[pr]};
      DevBuf* to[4] = {&b.links[pr], &b.cop[pr], &b.P[pr], &b.links_eo[pr]};
      for (int q = 0; q < 4; ++q) {
        if (!from[q]->p) continue;
        if (!to[q]->ensure(from[q]->bytes)) return MG_ENOMEM;
        CK(cudaMemcpyAsync(to[q]->p, from[q]->p, from[q]->bytes, cudaMemcpyDeviceToDevice, st));
      }
    }
    // A_l(m) = A_l(m0) + (m - m0) 1 on every coarse level (P^+ P = 1)
    if (l >= 1 && delta != 0.0) {
      LK(launch_diag_shift(b.cop[MG_F64].as<double2>(), b.ncomp, b.V, delta, st));
      const size_t ncop = (size_t)9 * b.ncomp * b.ncomp * b.V;
      for (int pr = 1; pr < 4; ++pr)
        if (b.cop[pr].p) LK(launch_convert(MG_F64, pr, ncop, 1, b.cop[MG_F64].p, b.cop[pr].p, 1.0, nullptr, 0, 0.0, 0, st));
    }
    if (a.cop_mma.p) {
      if (!b.cop_mma.ensure(a.cop_mma.bytes)) return MG_ENOMEM;
      LK(launch_mma_pack(b.cop[MG_F64].as<double2>(), b.ncomp, b.V, b.cop_mma.p, st));
    }
  }
  RET(ensure_reducer(h, 1));
  if (coarsest) RET(build_coarsest(h));
  CK(cudaStreamSynchronize(st));
  return MG_OK;
}

int mg_retarget(const mg_handle* src, double mass, mg_handle** hout, void* stream) {
  if (!hout) return MG_EINVAL;
  *hout = nullptr;
  if (!src) {
    set_error("mg_retarget: null handle");
    return MG_EINVAL;
  }
  mg_handle* h = new mg_handle();
  h->p = src->p;
  h->mass = mass;
  for (int m = 0; m < 4; ++m) h->dims[m] = src->dims[m];
  h->st = (cudaStream_t)stream;
  h->use_graphs = src->use_graphs;
  h->prof_mask = __atomic_load_n(&g_default_prof_mask, __ATOMIC_RELAXED);
  if ((h->host_slots = take_host_slots()) == nullptr) {
    cudaGetLastError();
    delete h;
    set_error("pinned host allocation failed");
    return MG_ENOMEM;
  }
  // the source's work must be complete before its buffers are copied
  if (src->st && src->st != h->st) cudaStreamSynchronize(src->st);
  int rc = retarget_impl(src, h);
  if (rc != MG_OK) {
    mg_destroy(h);
    return rc;
  }
  *hout = h;
  return MG_OK;
}

int mg_retarget_batch(const mg_handle* src, const double* masses, int count, mg_handle** hout, void* stream) {
  if (!hout || !masses || count < 1 || count > 64) {
    set_error("mg_retarget_batch: bad argument");
    return MG_EINVAL;
  }
  for (int z = 0; z < count; ++z) hout[z] = nullptr;
  if (!src) {
    set_error("mg_retarget_batch: null handle");
    return MG_EINVAL;
  }
  std::vector<mg_handle*> hs;
  auto fail = [&](int rc) {
    for (mg_handle* x : hs) mg_destroy(x);
    return rc;
  };
  if (src->st && src->st != (cudaStream_t)stream) cudaStreamSynchronize(src->st);
  for (int z = 0; z < count; ++z) {
    mg_handle* h = new mg_handle();
    h->p = src->p;
    h->mass = masses[z];
    for (int m = 0; m < 4; ++m) h->dims[m] = src->dims[m];
    h->st = (cudaStream_t)stream;
    h->use_graphs = src->use_graphs;
    h->prof_mask = __atomic_load_n(&g_default_prof_mask, __ATOMIC_RELAXED);
    hs.push_back(h);
    if ((h->host_slots = take_host_slots()) == nullptr) {
      cudaGetLastError();
      set_error("pinned host allocation failed");
      return fail(MG_ENOMEM);
    }
    const int rc = retarget_impl(src, h, false);
    if (rc != MG_OK) return fail(rc);
  }
  const int rc = build_coarsest_many(hs.data(), count);
  if (rc != MG_OK) return fail(rc);
  for (int z = 0; z < count; ++z) hout[z] = hs[z];
  return MG_OK;
}

int dslash_apply(mg_handle* h, int prec, const void* in, void* out, int nrhs, void* stream) {
  if (!h || !in || !out || nrhs < 1 || check_prec(prec)) {
    set_error("dslash_apply: bad argument");
    return MG_EINVAL;
  }
  cudaStream_t keep = h->st;
  h->st = (cudaStream_t)stream;
  int rc = ensure_reducer(h, nrhs);
  if (rc == MG_OK) rc = op_apply(h, 0, prec, in, out, nullptr, 1.0, 0.0, nullptr, 0, nrhs);
  h->st = keep;
  return rc;
}

static int eo_args_ok(mg_handle* h, int prec, int nrhs, const char* who) {
  if (!h || nrhs < 1 || check_prec(prec)) {
    set_error(std::string(who) + ": bad argument");
    return MG_EINVAL;
  }
  const Level& f = *h->lev[0];
  if (f.L[0] % 2 || f.L[1] % 2 || f.L[2] % 2 || f.L[3] % 2) {
    set_error(std::string(who) + ": every lattice extent must be even");
    return MG_EINVAL;
  }
  return MG_OK;
}

int eo_split(mg_handle* h, int prec, const void* full, void* even, void* odd, int nrhs, void* stream) {
  RET(eo_args_ok(h, prec, nrhs, "eo_split"));
  if (!full || !even || !odd) return MG_EINVAL;
  const Level& f = *h->lev[0];
  LK(launch_eo_split(4 * bytes_of(prec), full, even, odd, f.L, (size_t)3 * nrhs, (size_t)(f.V / 2),
                     (cudaStream_t)stream));
  return MG_OK;
}

int eo_merge(mg_handle* h, int prec, const void* even, const void* odd, void* full, int nrhs, void* stream) {
  RET(eo_args_ok(h, prec, nrhs, "eo_merge"));
  if (!full) return MG_EINVAL;
  const Level& f = *h->lev[0];
  LK(launch_eo_merge(prec, even, odd, full, f.L, (size_t)3 * nrhs, 0, (cudaStream_t)stream));
  return MG_OK;
}

int dslash_eo_apply(mg_handle* h, int prec, int parity_out, const void* x, const void* in, void* out, double a,
                    double b, int nrhs, void* stream) {
  RET(eo_args_ok(h, prec, nrhs, "dslash_eo_apply"));
  if (!in || !out || (parity_out != 0 && parity_out != 1)) {
    set_error("dslash_eo_apply: bad argument");
    return MG_EINVAL;
  }
  cudaStream_t keep = h->st;
  h->st = (cudaStream_t)stream;
  int rc = ensure_reducer(h, nrhs);
  if (rc == MG_OK) rc = eo_apply(h, prec, parity_out, x, in, nullptr, out, x ? a : 0.0, b, 0.0, nullptr, 0, nrhs);
  h->st = keep;
  return rc;
}

int schur_apply(mg_handle* h, int prec, const void* in, void* out, int nrhs, void* stream) {
  RET(eo_args_ok(h, prec, nrhs, "schur_apply"));
  if (!in || !out) return MG_EINVAL;
  cudaStream_t keep = h->st;
  h->st = (cudaStream_t)stream;
  int rc = ensure_reducer(h, nrhs);
  void* t = rc == MG_OK ? work(h, 0, prec, WV_EOB, nrhs) : nullptr;
  if (rc == MG_OK && !t) rc = MG_ENOMEM;
  if (rc == MG_OK) rc = schur_op(h, prec, in, out, t, nullptr, nullptr, 0, nrhs);
  h->st = keep;
  return rc;
}

int coarse_apply(mg_handle* h, int level, int prec, const void* in, void* out, int nrhs, void* stream) {
  if (!h || level < 1 || level >= (int)h->lev.size() || !in || !out || nrhs < 1 || check_prec(prec)) {
    set_error("coarse_apply: bad argument");
    return MG_EINVAL;
  }
  cudaStream_t keep = h->st;
  h->st = (cudaStream_t)stream;
  int rc = ensure_reducer(h, nrhs);
  if (rc == MG_OK) rc = op_apply(h, level, prec, in, out, nullptr, 1.0, 0.0, nullptr, 0, nrhs);
  h->st = keep;
  return rc;
}

int restrict_apply(mg_handle* h, int level, int prec, const void* in, void* out, int nrhs, void* stream) {
  if (!h || level < 0 || level + 1 >= (int)h->lev.size() || !in || !out || nrhs < 1 || check_prec(prec) ||
      !h->lev[level]->P[prec].p) {
    set_error("restrict_apply: bad argument or prolongator not stored in this precision");
    return MG_EINVAL;
  }
  Level& a = *h->lev[level];
  const int pout = prec == MG_F64 ? MG_F64 : MG_F32;
  LK(launch_restrict(prec, prec, pout, agg_of(a), a.P[prec].p, in, out, nrhs, (cudaStream_t)stream));
  return MG_OK;
}

int prolong_apply(mg_handle* h, int level, int prec, const void* in, void* out, int nrhs, void* stream) {
  if (!h || level < 0 || level + 1 >= (int)h->lev.size() || !in || !out || nrhs < 1 || check_prec(prec) ||
      !h->lev[level]->P[prec].p) {
    set_error("prolong_apply: bad argument or prolongator not stored in this precision");
    return MG_EINVAL;
  }
  Level& a = *h->lev[level];
  const int pin = prec == MG_F64 ? MG_F64 : MG_F32;
  LK(launch_prolong(pin, prec, prec, agg_of(a), a.P[prec].p, in, out, nrhs, (cudaStream_t)stream));
  return MG_OK;
}

int mr_apply(mg_handle* h, int level, int prec, const void* b, void* x, void* r, int steps, void* stream) {
  if (!h || level < 0 || level >= (int)h->lev.size() || !b || !x || !r || steps < 0 || check_prec(prec)) {
    set_error("mr_apply: bad argument");
    return MG_EINVAL;
  }
  cudaStream_t keep = h->st;
  h->st = (cudaStream_t)stream;
  int rc = ensure_reducer(h, 1);
  if (rc == MG_OK) rc = op_apply(h, level, prec, x, r, b, -1.0, 1.0, nullptr, 0, 1);
  if (rc == MG_OK) rc = mr_steps(h, level, prec, b, x, false, r, steps, 1);
  h->st = keep;
  return rc;
}

int vcycle_apply(mg_handle* h, const void* r, void* e, void* stream) {
  if (!h || !r || !e || h->lev.size() < 2 || h->p.mixed) {
    set_error("vcycle_apply: needs a plain FP64 hierarchy with >= 2 levels");
    return MG_EINVAL;
  }
  cudaStream_t keep = h->st;
  h->st = (cudaStream_t)stream;
  int rc = ensure_reducer(h, 1);
  if (rc == MG_OK) rc = ensure_coarsest(h);
  if (rc == MG_OK) rc = vcycle(h, 0, r, e, 1);
  h->st = keep;
  return rc;
}

int mg_field_to_internal(mg_handle* h, int level, int prec, const double* ext, int on_device, void* internal,
                         int nrhs, void* stream) {
  if (!h || level < 0 || level >= (int)h->lev.size() || !ext || !internal || nrhs < 1 || check_prec(prec)) {
    set_error("mg_field_to_internal: bad argument");
    return MG_EINVAL;
  }
  Level& a = *h->lev[level];
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf tmp;
  const void* src = ext;
  if (!on_device) {
    if (!tmp.ensure(a.n() * nrhs * 16)) return MG_ENOMEM;
    CK(cudaMemcpyAsync(tmp.p, ext, a.n() * nrhs * 16, cudaMemcpyHostToDevice, st));
    src = tmp.p;
  }
  LK(launch_ext_to_int(prec, a.ncomp, a.q, a.V, nrhs, src, internal, st));
  if (!on_device) CK(cudaStreamSynchronize(st));
  return MG_OK;
}

int mg_field_from_internal(mg_handle* h, int level, int prec, const void* internal, double* ext, int on_device,
                           int nrhs, void* stream) {
  if (!h || level < 0 || level >= (int)h->lev.size() || !ext || !internal || nrhs < 1 || check_prec(prec)) {
    set_error("mg_field_from_internal: bad argument");
    return MG_EINVAL;
  }
  Level& a = *h->lev[level];
  cudaStream_t st = (cudaStream_t)stream;
  if (on_device) {
    LK(launch_int_to_ext(prec, a.ncomp, a.q, a.V, nrhs, internal, ext, st));
    return MG_OK;
  }
  DevBuf tmp;
  if (!tmp.ensure(a.n() * nrhs * 16)) return MG_ENOMEM;
  LK(launch_int_to_ext(prec, a.ncomp, a.q, a.V, nrhs, internal, tmp.p, st));
  CK(cudaMemcpyAsync(ext, tmp.p, a.n() * nrhs * 16, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return MG_OK;
}

int mg_level_info(mg_handle* h, int level, int dims_out[4], int* ncomp, int* nv) {
  if (!h || level < 0 || level >= (int)h->lev.size()) return MG_EINVAL;
  Level& a = *h->lev[level];
  if (dims_out)
    for (int m = 0; m < 4; ++m) dims_out[m] = a.L[m];
  if (ncomp) *ncomp = a.ncomp;
  if (nv) *nv = a.nv;
  return MG_OK;
}

int mg_get_prolongator(mg_handle* h, int level, double* out) {
  if (!h || level < 0 || level + 1 >= (int)h->lev.size() || !out) return MG_EINVAL;
  Level& a = *h->lev[level];
  cudaStream_t st = h->st;
  DevBuf f, tot, ext;
  if (!f.ensure(a.n() * 16) || !tot.ensure(a.n() * 16) || !ext.ensure(a.n() * 16)) return MG_ENOMEM;
  const Agg g = agg_of(a);
  for (int k = 0; k < a.nv; ++k) {
    LK(launch_p_column(MG_F64, g, a.P[MG_F64].p, k, 1, tot.p, st));
    LK(launch_p_column(MG_F64, g, a.P[MG_F64].p, a.nv + k, 1, f.p, st));
    LK(launch_convert(MG_F64, MG_F64, a.n(), 1, f.p, tot.p, 1.0, nullptr, 0, 0.0, 1, st));
    LK(launch_int_to_ext(MG_F64, a.ncomp, a.q, a.V, 1, tot.p, ext.p, st));
    CK(cudaMemcpyAsync(out + (size_t)k * a.n() * 2, ext.p, a.n() * 16, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  return MG_OK;
}

int mg_get_coarse_op(mg_handle* h, int level, double* out) {
  if (!h || level < 1 || level >= (int)h->lev.size() || !out) return MG_EINVAL;
  Level& a = *h->lev[level];
  const size_t n = a.ncomp, V = a.V;
  std::vector<double> tmp((size_t)9 * n * n * V * 2);
  CK(cudaMemcpyAsync(tmp.data(), a.cop[MG_F64].p, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  // [9][i][j][B] -> [9][B][i][j]
  for (size_t d = 0; d < 9; ++d)
    for (size_t i = 0; i < n; ++i)
      for (size_t j = 0; j < n; ++j)
        for (size_t B = 0; B < V; ++B) {
          const size_t src = (((d * n + i) * n + j) * V + B) * 2;
          const size_t dst = (((d * V + B) * n + i) * n + j) * 2;
          out[dst] = tmp[src];
          out[dst + 1] = tmp[src + 1];
        }
  return MG_OK;
}

int mg_get_coarsest_inverse(mg_handle* h, double* out) {
  if (!h || h->lev.size() < 2 || !out) return MG_EINVAL;
  if (h->lev.back()->inv_pending) RET(build_coarsest(h));
  Level& c = *h->lev.back();
  const size_t n = c.ncomp, V = c.V, N = n * V;
  const bool f64 = c.inv_prec == MG_F64;
  std::vector<double> d(f64 ? N * N * 2 : 0);
  std::vector<float> f(f64 ? 0 : N * N * 2);
  if (f64)
    CK(cudaMemcpyAsync(d.data(), c.inv.p, d.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  else
    CK(cudaMemcpyAsync(f.data(), c.inv.p, f.size() * sizeof(float), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  // internal order (i V + B) -> external order (B n + i), rows and columns
  for (size_t i = 0; i < n; ++i)
    for (size_t B = 0; B < V; ++B)
      for (size_t j = 0; j < n; ++j)
        for (size_t Bp = 0; Bp < V; ++Bp) {
          const size_t src = ((i * V + B) * N + j * V + Bp) * 2;
          const size_t dst = ((B * n + i) * N + Bp * n + j) * 2;
          out[dst] = f64 ? d[src] : (double)f[src];
          out[dst + 1] = f64 ? d[src + 1] : (double)f[src + 1];
        }
  return MG_OK;
}

unsigned long long mg_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

unsigned long long mg_alloc_count(void) { return wmg::g_dev_allocs.load(std::memory_order_relaxed); }

int mg_tune(int mode) {
  if (mode < 0 || mode > 4) return -1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const int prev = g_tune_mode;
  if (mode == 2) {
    g_tune.clear();
    g_tune_mode = 1;
  } else {
    g_tune_mode = mode;
  }
  return prev;
}

int mg_tune_report(char* buf, int cap) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string r;
  for (auto& kv : g_tune) {
    r += kv.first + " " + std::to_string(kv.second.variant);
    for (float u : kv.second.us) r += " " + std::to_string(u);
    r += "\n";
  }
  if (buf && cap > 0) {
    const size_t n = std::min(r.size(), (size_t)cap - 1);
    memcpy(buf, r.data(), n);
    buf[n] = 0;
  }
  return (int)r.size();
}

int mg_profile(mg_handle* h, unsigned mask) {
  if (!h) {
    __atomic_store_n(&g_default_prof_mask, mask, __ATOMIC_RELAXED);
    return MG_OK;
  }
  CK(cudaStreamSynchronize(h->st));
  h->prof_marks.clear();
  h->prof_used = 0;
  h->prof_mask = mask;
  return MG_OK;
}

int mg_profile_bytes(mg_handle* h, int kclass, int prec, double* bytes) {
  if (!h || !bytes || kclass < 0 || kclass >= MG_K_CLASSES || check_prec(prec)) return MG_EINVAL;
  double tot = 0.0;
  for (auto& m : h->prof_marks)
    if (m.key == kclass * 4 + prec) tot += m.bytes;
  *bytes = tot;
  return MG_OK;
}

int mg_profile_read(mg_handle* h, int kclass, int prec, long long* launches, double* ms) {
  if (!h || kclass < 0 || kclass >= MG_K_CLASSES || check_prec(prec)) return MG_EINVAL;
  CK(cudaStreamSynchronize(h->st));
  long long n = 0;
  double tot = 0.0;
  for (auto& m : h->prof_marks) {
    if (m.key != kclass * 4 + prec) continue;
    CK(cudaEventSynchronize(h->prof_pool[m.idx + 1]));
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, h->prof_pool[m.idx], h->prof_pool[m.idx + 1]));
    tot += t;
    ++n;
  }
  if (launches) *launches = n;
  if (ms) *ms = tot;
  return MG_OK;
}

size_t mg_footprint(const int dims[4], const mg_params* p, int nrhs) {
  if (!dims || !p) return 0;
  size_t V = (size_t)dims[0] * dims[1] * dims[2] * dims[3];
  size_t bytes = (size_t)4 * V * 9 * 16 * 2;                      // links + upload staging
  const size_t vec = V * 12 * 16;                                  // one FP64 fine vector
  bytes += vec * (size_t)nrhs * (2 * (size_t)p->gcr_restart + 8);  // GCR basis + work
  size_t Vl = V, nc = 12;
  for (int l = 0; l + 1 < p->n_levels; ++l) {
    size_t bs = (size_t)p->block[l][0] * p->block[l][1] * p->block[l][2] * p->block[l][3];
    bytes += Vl * nc * 16 * (size_t)p->nv[l] * 4;  // candidates, relaxation work, P
    Vl /= bs;
    nc = 2 * (size_t)p->nv[l];
    bytes += 9 * nc * nc * Vl * 16 * 2;            // coarse stencil
    bytes += Vl * nc * 16 * (size_t)nrhs * 10;     // coarse work vectors
  }
  if (p->n_levels >= 2) {
    const size_t N2 = (Vl * nc) * (Vl * nc);
    bytes += N2 * 16 * 3;  // dense inverse + elimination scratch
    if (nrhs > 1) bytes += N2 * (p->mixed ? 8 : 16) * 3 * (size_t)nrhs;  // mg_solve_masses: one per mass
  }
  return bytes;
}

}  // extern "C"

// ====================================================================== solve
namespace {

int gcr_solve(mg_handle* h, const double* b_ext, double* x_ext, int nrhs, int on_device, double tol,
              mg_stats* stats) {
  cudaStream_t st = h->st;
  Level& f = *h->lev[0];
  const size_t n = f.n();
  const bool mixed = h->p.mixed != 0;
  const int pin = mixed ? MG_F32 : MG_F64;   // inner (Krylov) precision
  const size_t bi = bytes_of(pin);
  const int restart = h->p.gcr_restart;
  RET(ensure_reducer(h, nrhs));
  if (!h->mm_active) RET(ensure_coarsest(h));  // a mass per right-hand side uses the inverses of its masses
  auto t0 = std::chrono::steady_clock::now();
  // FP64 x, b, r in the internal layout
  if (!h->gx64.ensure(n * nrhs * 16) || !h->gb64.ensure(n * nrhs * 16) || !h->gr64.ensure(n * nrhs * 16) ||
      !h->gtmp.ensure(n * nrhs * 16))
    return MG_ENOMEM;
  {
    const void* bsrc = b_ext;
    const void* xsrc = x_ext;
    DevBuf stage;
    if (!on_device) {
      if (!stage.ensure(n * nrhs * 16 * 2)) return MG_ENOMEM;
      CK(cudaMemcpyAsync(stage.p, b_ext, n * nrhs * 16, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync((char*)stage.p + n * nrhs * 16, x_ext, n * nrhs * 16, cudaMemcpyHostToDevice, st));
      bsrc = stage.p;
      xsrc = (char*)stage.p + n * nrhs * 16;
    }
    LK(launch_ext_to_int(MG_F64, 12, 4, f.V, nrhs, bsrc, h->gb64.p, st));
    LK(launch_ext_to_int(MG_F64, 12, 4, f.V, nrhs, xsrc, h->gx64.p, st));
    CK(cudaStreamSynchronize(st));
    stage.release_idle();
  }
  // Krylov buffers in precision pin: basis W, Z [restart][nrhs][n], x, r
  const size_t vbytes = n * nrhs * bi;
  const size_t slots = (size_t)((restart + 7) / 8) * 8;  // the multi-dot reads whole chunks of 8
  const size_t hbytes = (size_t)nrhs * kMaxBasis * kMaxBasis * 16, abytes = (size_t)nrhs * kMaxBasis * 16;
  if (!h->gW.ensure(vbytes * slots) || !h->gZ.ensure(vbytes * restart) || !h->gr.ensure(vbytes) ||
      !h->gH.ensure(hbytes) || !h->galpha.ensure(abytes) || !h->gy.ensure(abytes))
    return MG_ENOMEM;
  double2* H = h->gH.as<double2>();
  double2* alpha = h->galpha.as<double2>();
  double* hs = h->host_slots;
  std::vector<double> bn(nrhs), rn(nrhs);
  LK(launch_dot(MG_F64, n, nrhs, h->gb64.p, h->gb64.p, h->red.at(slot_gcr_bn(), 4), st));
  RET(read_slots(h, slot_gcr_bn(), 4 * nrhs));
  for (int r = 0; r < nrhs; ++r) bn[r] = sqrt(hs[4 * r + 2]);
  for (int r = 0; r < nrhs; ++r)
    if (bn[r] == 0.0) {
      set_error("mg_solve: zero right-hand side");
      return MG_EINVAL;
    }
  std::vector<int> iters(nrhs, 0), done(nrhs, 0);
  int restarts = 0, reliable = 0, status = MG_OK;
  long long fine = 0, fine64 = 0;
  const long long per_cycle = (h->lev.size() >= 2) ? (h->p.nu_pre + h->p.nu_post + 1) : 0;
  int total_iters = 0;
  // true residual r64 = b - D x64 (FP64)
  auto true_residual = [&]() -> int {
    RET(op_apply(h, 0, MG_F64, h->gx64.p, h->gr64.p, h->gb64.p, -1.0, 1.0, nullptr, 0, nrhs));
    ++fine;
    ++fine64;
    LK(launch_dot(MG_F64, n, nrhs, h->gr64.p, h->gr64.p, h->red.at(slot_gcr_rn(), 4), st));
    RET(read_slots(h, slot_gcr_rn(), 4 * nrhs));
    for (int r = 0; r < nrhs; ++r) rn[r] = sqrt(h->host_slots[4 * r + 2]);
    return MG_OK;
  };
  RET(true_residual());
  bool all_done = true;
  for (int r = 0; r < nrhs; ++r) {
    if (!isfinite(rn[r])) return MG_ENAN;
    done[r] = rn[r] <= tol * bn[r];
    all_done &= (bool)done[r];
  }
  while (!all_done) {
    if (total_iters >= h->p.max_iter) {
      status = MG_ENOCONV;
      break;
    }
    // start of a cycle: Krylov residual r = r64 (converted), H = 0
    LK(launch_convert(MG_F64, pin, n, nrhs, h->gr64.p, h->gr.p, 1.0, nullptr, 0, 0.0, 0, st));
    CK(cudaMemsetAsync(H, 0, hbytes, st));
    LK(launch_dot(pin, n, nrhs, h->gr.p, h->gr.p, h->red.at(slot_gcr_rn(), 4), st));
    std::vector<double> r0 = rn;
    int k = 0;
    for (;;) {
      char* zk = (char*)h->gZ.p + (size_t)k * vbytes;
      char* wk = (char*)h->gW.p + (size_t)k * vbytes;
      // z = M r
      if (h->lev.size() >= 2) {
        const int pf = prec_of(h, 0);
        if (pf == pin) {
          void* eout = work(h, 0, pf, WV_A, nrhs);
          if (!eout) return MG_ENOMEM;
          RET(vcycle_graph(h, h->gr.p, eout, nrhs));
          CK(cudaMemcpyAsync(zk, eout, vbytes, cudaMemcpyDeviceToDevice, st));
        } else {
          void* rin = work(h, 0, pf, WV_IN, nrhs);
          void* eout = work(h, 0, pf, WV_A, nrhs);
          if (!rin || !eout) return MG_ENOMEM;
          // scale the residual to RMS 1/8 per component for 16-bit storage
          const double sig = sqrt((double)n) / 8.0;
          const double cvb = (double)n * nrhs * (bytes_of(pin) + bytes_of(pf));
          {
            Prof pf2(h, MG_K_VECTOR, pin, cvb);
            LK(launch_convert(pin, pf, n, nrhs, h->gr.p, rin, sig, h->red.slot(slot_gcr_rn() + 2), 4, -0.5, 0, st));
          }
          RET(vcycle_graph(h, rin, eout, nrhs));
          Prof pf2(h, MG_K_VECTOR, pin, cvb);
          LK(launch_convert(pf, pin, n, nrhs, eout, zk, 1.0 / sig, h->red.slot(slot_gcr_rn() + 2), 4, 0.5, 0, st));
        }
        fine += per_cycle;
      } else {
        CK(cudaMemcpyAsync(zk, h->gr.p, vbytes, cudaMemcpyDeviceToDevice, st));
      }
      // w = D z, with <w|r> and ||w||^2 fused
      RET(op_apply(h, 0, pin, zk, wk, nullptr, 1.0, 0.0, h->gr.p, slot_gcr_pre(), nrhs));
      ++fine;
      if (pin == MG_F64) ++fine64;
      // classical Gram-Schmidt of w against the previous w's (z stays as the
      // cycle made it): one pass, and a second one for the right-hand sides
      // whose ||w|| the first pass cut below 1/sqrt(2)
      const double* dots = h->red.slot(slot_gcr_pre());
      if (k > 0) {
        // one pass: the multi-dot reads W_0..W_k-1 and w, the update reads them and r and writes w
        Prof pf2(h, MG_K_GRAM, pin, (2.0 * k + 4.0) * (double)vbytes);
        for (int pass = 0; pass < 2; ++pass) {
          const double* pre = pass ? h->red.slot(slot_gcr_pre() + 2) : nullptr;
          const double* post = pass ? h->red.slot(slot_gcr_wr() + 2) : nullptr;
          LK(launch_multidot(pin, n, nrhs, k, kMaxBasis, h->gW.p, n * nrhs, wk, h->red.at(slot_beta(), 0), st, pre,
                             post, 4));
          LK(launch_gs_update(pin, n, nrhs, k, kMaxBasis, h->red.slot(slot_beta()), h->gW.p, n * nrhs, wk, h->gr.p,
                              h->red.at(slot_gcr_wr(), 4), H, k, pre, post, 4, st));
        }
        dots = h->red.slot(slot_gcr_wr());
      }
      {
        Prof pf2(h, MG_K_VECTOR, pin, 4.0 * (double)vbytes);
        LK(launch_gcr_step(pin, n, nrhs, dots, 4, wk, h->gr.p, h->red.at(slot_gcr_rn() + 2, 4), H, alpha, k,
                           kMaxBasis, st));
      }
      RET(read_slots(h, slot_gcr_rn(), 4 * nrhs));
      ++k;
      ++total_iters;
      bool inner_done = true;
      for (int r = 0; r < nrhs; ++r) {
        const double v = sqrt(hs[4 * r + 2]);
        if (!isfinite(v)) {
          set_error("mg_solve: residual norm is not finite");
          return MG_ENAN;
        }
        if (!done[r]) ++iters[r];
        const double target = mixed ? std::max(tol * bn[r] * 0.5, h->p.reliable_delta * r0[r]) : tol * bn[r];
        if (!done[r] && v > target) inner_done = false;
      }
      if (inner_done || k == restart || total_iters >= h->p.max_iter) break;
    }
    // x64 += Z H^-1 alpha (the cycle's correction), then the true residual in FP64
    {
      Prof pf2(h, MG_K_VECTOR, pin, (double)k * vbytes + 2.0 * n * nrhs * 16);
      LK(launch_back_substitute(nrhs, k, kMaxBasis, H, alpha, h->gy.as<double2>(), st));
      LK(launch_zcombine(pin, MG_F64, n, nrhs, k, kMaxBasis, h->gy.as<double2>(), h->gZ.p, n * nrhs, h->gx64.p, st));
    }
    RET(true_residual());
    if (k == restart) ++restarts;
    ++reliable;
    all_done = true;
    for (int r = 0; r < nrhs; ++r) {
      if (!isfinite(rn[r])) {
        set_error("mg_solve: true residual is not finite");
        return MG_ENAN;
      }
      if (!done[r] && rn[r] <= tol * bn[r]) done[r] = 1;
      all_done &= (bool)done[r];
    }
  }
  // result back to the external layout
  {
    DevBuf stage;
    void* dst = x_ext;
    if (!on_device) {
      if (!stage.ensure(n * nrhs * 16)) return MG_ENOMEM;
      dst = stage.p;
    }
    LK(launch_int_to_ext(MG_F64, 12, 4, f.V, nrhs, h->gx64.p, dst, st));
    if (!on_device) CK(cudaMemcpyAsync(x_ext, stage.p, n * nrhs * 16, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    stage.release_idle();
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) {
    for (int r = 0; r < nrhs; ++r) {
      stats[r].iters = iters[r];
      stats[r].restarts = restarts;
      stats[r].reliable_updates = reliable;
      stats[r].fine_dslash = fine;
      stats[r].fine_dslash_f64 = fine64;
      stats[r].true_rel_residual = rn[r] / bn[r];
      stats[r].solve_seconds = secs;
    }
  }
  return status;
}

}  // namespace

// ====================================================================== Krylov baselines
namespace {

// A level-0 FP64 system for the Krylov baselines: the full operator D on
// level-0 fields, or the even-odd Schur complement S on half fields (both in
// the chunked layout; n = 12 x sites).  Both are gamma5-Hermitian (Sec. 1).
struct KSys {
  size_t n;                                                     // complex elements of a vector
  std::function<int(const void* in, void* out)> apply;          // out = A in
  std::function<int(const void* x, void* r, const void* b)> resid;  // r = b - A x
};

// out = A^+ in = gamma5 A gamma5 in: the chirality - components change sign before and after A.
int apply_dag(mg_handle* h, const KSys& sys, const void* in, void* out, void* tmp) {
  const size_t sites = sys.n / 12;
  LK(launch_gamma5(sites, 1, in, tmp, h->st));
  RET(sys.apply(tmp, out));
  LK(launch_gamma5(sites, 1, out, out, h->st));
  return MG_OK;
}

struct Cx {
  double re, im;
};
inline Cx cdiv(Cx a, Cx b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
inline Cx cmul(Cx a, Cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// out = c0 x0 + c1 x1 + c2 x2, with <w|out>, ||out||^2 into slot (w optional)
int lincomb(mg_handle* h, size_t n, double2* out, std::initializer_list<std::pair<const void*, Cx>> terms,
            const void* w, size_t slot) {
  LinComb L;
  L.out = out;
  L.w = (const double2*)w;
  int t = 0;
  for (auto& tc : terms) {
    L.x[t] = (const double2*)tc.first;
    L.c[t] = make_double2(tc.second.re, tc.second.im);
    ++t;
  }
  for (; t < 3; ++t) {
    L.x[t] = nullptr;
    L.c[t] = make_double2(0.0, 0.0);
  }
  Prof pf(h, MG_K_VECTOR, MG_F64, (double)n * 16 * (terms.size() + 1 + (w != nullptr)));
  LK(launch_lincomb(n, L, h->red.at(slot, 4), h->st));
  return MG_OK;
}

// <a|b>, ||a||^2, ||b||^2 of two FP64 vectors of n elements, read back
int dot3(mg_handle* h, size_t n, const void* a, const void* b, Cx* ab, double* aa, double* bb) {
  {
    Prof pf(h, MG_K_VECTOR, MG_F64, (double)n * 16 * (a == b ? 1 : 2));
    LK(launch_dot(MG_F64, n, 1, a, b, h->red.at(slot_misc(), 4), h->st));
  }
  RET(read_slots(h, slot_misc(), 4));
  const double* s = h->host_slots;
  if (ab) *ab = {s[0], s[1]};
  if (aa) *aa = s[2];
  if (bb) *bb = s[3];
  return MG_OK;
}

int krylov_one(mg_handle* h, const KSys& sys, int method, double2* b, double2* x, double tol, int max_iter,
               mg_stats* st) {
  const size_t n = sys.n, vb = n * 16;
  DevBuf buf;
  if (!buf.ensure(vb * 6)) return MG_ENOMEM;
  double2* r = buf.as<double2>();
  double2* v1 = r + n;  // BiCGstab: rhat | CGNR: z
  double2* v2 = r + 2 * n;  // p
  double2* v3 = r + 3 * n;  // v | q
  double2* v4 = r + 4 * n;  // s | D^+ scratch
  double2* v5 = r + 5 * n;  // t
  long long mv = 0;
  int iters = 0;
  double bb = 0.0, rr = 0.0;
  RET(dot3(h, n, b, b, nullptr, &bb, nullptr));
  const double bn = sqrt(bb);
  if (!(bn > 0.0)) {
    set_error("krylov_solve: zero right-hand side");
    return MG_EINVAL;
  }
  int status = MG_ENOCONV;
  const size_t sl = slot_misc() + 4;
  while (iters < max_iter) {
    RET(sys.resid(x, r, b));  // r = b - A x
    ++mv;
    RET(dot3(h, n, r, r, nullptr, &rr, nullptr));
    if (!isfinite(rr)) {
      set_error("krylov_solve: residual is not finite");
      return MG_ENAN;
    }
    if (sqrt(rr) <= tol * bn) {
      status = MG_OK;
      break;
    }
    if (method == MG_KRYLOV_BICGSTAB) {
      CK(cudaMemcpyAsync(v1, r, vb, cudaMemcpyDeviceToDevice, h->st));  // shadow residual
      CK(cudaMemsetAsync(v2, 0, vb, h->st));
      CK(cudaMemsetAsync(v3, 0, vb, h->st));
      Cx rho = {1, 0}, alpha = {1, 0}, omega = {1, 0}, rho_new = {rr, 0};
      while (iters < max_iter) {
        const Cx beta = cmul(cdiv(rho_new, rho), cdiv(alpha, omega));
        const Cx bo = cmul(beta, omega);
        RET(lincomb(h, n, v2, {{r, {1, 0}}, {v2, beta}, {v3, {-bo.re, -bo.im}}}, nullptr, sl));  // p
        RET(sys.apply(v2, v3));  // v = A p
        ++mv;
        Cx rv;
        RET(dot3(h, n, v1, v3, &rv, nullptr, nullptr));
        alpha = cdiv(rho_new, rv);
        RET(lincomb(h, n, v4, {{r, {1, 0}}, {v3, {-alpha.re, -alpha.im}}}, v1, sl));  // s = r - alpha v
        RET(read_slots(h, sl, 4));
        ++iters;
        if (sqrt(h->host_slots[2]) <= tol * bn) {  // converged on the half step
          RET(lincomb(h, n, x, {{x, {1, 0}}, {v2, alpha}}, nullptr, sl));
          break;
        }
        RET(sys.apply(v4, v5));  // t = A s
        ++mv;
        Cx ts;
        double tt = 0.0;
        RET(dot3(h, n, v5, v4, &ts, &tt, nullptr));
        omega = {ts.re / tt, ts.im / tt};
        RET(lincomb(h, n, x, {{x, {1, 0}}, {v2, alpha}, {v4, omega}}, nullptr, sl));          // x += alpha p + omega s
        RET(lincomb(h, n, r, {{v4, {1, 0}}, {v5, {-omega.re, -omega.im}}}, v1, sl));          // r = s - omega t
        RET(read_slots(h, sl, 4));
        rho = rho_new;
        rho_new = {h->host_slots[0], h->host_slots[1]};
        const double rn = sqrt(h->host_slots[2]);
        if (!isfinite(rn)) {
          set_error("krylov_solve: residual is not finite");
          return MG_ENAN;
        }
        if (rn <= tol * bn) break;
      }
    } else {
      RET(apply_dag(h, sys, r, v1, v4));  // z = A^+ r
      ++mv;
      CK(cudaMemcpyAsync(v2, v1, vb, cudaMemcpyDeviceToDevice, h->st));
      double zz = 0.0;
      RET(dot3(h, n, v1, v1, nullptr, &zz, nullptr));
      while (iters < max_iter) {
        RET(sys.apply(v2, v3));  // q = A p
        ++mv;
        double qq = 0.0;
        RET(dot3(h, n, v3, v3, nullptr, &qq, nullptr));
        const double a = zz / qq;
        RET(lincomb(h, n, x, {{x, {1, 0}}, {v2, {a, 0}}}, nullptr, sl));
        RET(lincomb(h, n, r, {{r, {1, 0}}, {v3, {-a, 0}}}, r, sl));
        RET(read_slots(h, sl, 4));
        ++iters;
        const double rn = sqrt(h->host_slots[2]);
        if (!isfinite(rn)) {
          set_error("krylov_solve: residual is not finite");
          return MG_ENAN;
        }
        if (rn <= tol * bn) break;
        RET(apply_dag(h, sys, r, v1, v4));
        ++mv;
        double zn = 0.0;
        RET(dot3(h, n, v1, v1, nullptr, &zn, nullptr));
        RET(lincomb(h, n, v2, {{v1, {1, 0}}, {v2, {zn / zz, 0}}}, nullptr, sl));
        zz = zn;
      }
    }
  }
  if (status != MG_OK) {  // the true residual at exit
    RET(sys.resid(x, r, b));
    ++mv;
    RET(dot3(h, n, r, r, nullptr, &rr, nullptr));
    if (sqrt(rr) <= tol * bn) status = MG_OK;
  }
  if (st) {
    st->iters = iters;
    st->restarts = 0;
    st->reliable_updates = 0;
    st->fine_dslash = mv;
    st->fine_dslash_f64 = mv;
    st->true_rel_residual = sqrt(rr) / bn;
  }
  return status;
}

// One right-hand side through the even-odd Schur system (FP64): b^_e = b_e +
// H_eo b_o / (2M), the Krylov method on S x_e = b^_e, x_o = (b_o + H_oe x_e / 2) / M.
// The full residual of the reconstructed x equals the Schur residual (exactly,
// up to rounding), so the Schur solve stops at tol ||b||; if rounding leaves the
// full true residual above tol ||b||, the Schur solve continues with a tighter
// target (at most 3 times).
int krylov_eo_one(mg_handle* h, int method, double2* b, double2* x, double tol, int max_iter, mg_stats* st) {
  Level& f = *h->lev[0];
  const size_t n = f.n(), nh = n / 2;
  const double M = 4.0 + h->mass;
  DevBuf buf;
  if (!buf.ensure(nh * 16 * 6 + n * 16)) return MG_ENOMEM;
  double2* be = buf.as<double2>();
  double2* bo = be + nh;
  double2* bh = bo + nh;
  double2* xe = bh + nh;
  double2* xo = xe + nh;
  double2* t = xo + nh;
  double2* rf = t + nh;  // full residual
  KSys sys;
  sys.n = nh;
  sys.apply = [&](const void* in, void* out) { return schur_op(h, MG_F64, in, out, t, nullptr, nullptr, 0, 1); };
  sys.resid = [&](const void* xx, void* r, const void* bb) {
    return schur_op(h, MG_F64, xx, r, t, bb, nullptr, 0, 1);
  };
  LK(launch_eo_split(64, b, be, bo, f.L, 3, nh / 12, h->st));
  LK(launch_eo_split(64, x, xe, xo, f.L, 3, nh / 12, h->st));
  RET(eo_apply(h, MG_F64, 0, be, bo, nullptr, bh, 1.0, 1.0 / (2.0 * M), 0.0, nullptr, 0, 1));
  double b2 = 0.0, bh2 = 0.0;
  RET(dot3(h, n, b, b, nullptr, &b2, nullptr));
  RET(dot3(h, nh, bh, bh, nullptr, &bh2, nullptr));
  const double bn = sqrt(b2);
  if (!(bn > 0.0) || !(bh2 > 0.0)) {
    set_error("krylov_solve: zero right-hand side");
    return MG_EINVAL;
  }
  double target = tol * bn / sqrt(bh2);
  long long mv = 1;  // the two half hops of b^_e and x_o
  int iters = 0, status = MG_ENOCONV;
  double rel = 0.0;
  for (int attempt = 0; attempt < 4; ++attempt) {
    mg_stats s1;
    const int s = krylov_one(h, sys, method, bh, xe, target, max_iter - iters, &s1);
    if (s != MG_OK && s != MG_ENOCONV) return s;
    iters += s1.iters;
    mv += s1.fine_dslash;
    RET(eo_apply(h, MG_F64, 1, bo, xe, nullptr, xo, 1.0 / M, 1.0 / (2.0 * M), 0.0, nullptr, 0, 1));
    LK(launch_eo_merge(MG_F64, xe, xo, x, f.L, 3, 0, h->st));
    RET(op_apply(h, 0, MG_F64, x, rf, b, -1.0, 1.0, nullptr, 0, 1));  // the full true residual
    ++mv;
    double r2 = 0.0;
    RET(dot3(h, n, rf, rf, nullptr, &r2, nullptr));
    rel = sqrt(r2) / bn;
    if (!isfinite(rel)) {
      set_error("krylov_solve: residual is not finite");
      return MG_ENAN;
    }
    if (rel <= tol) {
      status = MG_OK;
      break;
    }
    if (s == MG_ENOCONV || iters >= max_iter) break;
    target *= 0.5 * tol / rel;
  }
  if (st) {
    st->iters = iters;
    st->restarts = 0;
    st->reliable_updates = 0;
    st->fine_dslash = mv;
    st->fine_dslash_f64 = mv;
    st->true_rel_residual = rel;
  }
  return status;
}

}  // namespace

extern "C" int krylov_solve(mg_handle* h, int method, const double* b_ext, double* x_ext, int nrhs, int on_device,
                            double tol, int max_iter, mg_stats* stats, void* stream) {
  const bool eo = method == MG_KRYLOV_BICGSTAB_EO || method == MG_KRYLOV_CGNR_EO;
  if (!h || !b_ext || !x_ext || nrhs < 1 || !(tol > 0.0) || max_iter < 1 || method < 0 ||
      method > MG_KRYLOV_CGNR_EO || !h->lev[0]->links[MG_F64].p) {
    set_error("krylov_solve: bad argument");
    return MG_EINVAL;
  }
  const Level& f0 = *h->lev[0];
  if (eo && (f0.L[0] % 2 || f0.L[1] % 2 || f0.L[2] % 2 || f0.L[3] % 2)) {
    set_error("krylov_solve: the even-odd methods need every lattice extent even");
    return MG_EINVAL;
  }
  const int base = eo ? method - MG_KRYLOV_BICGSTAB_EO : method;
  cudaStream_t keep = h->st;
  h->st = (cudaStream_t)stream;
  Level& f = *h->lev[0];
  const size_t n = f.n(), vb = n * 16;
  int rc = MG_OK;
  DevBuf bx, stage;
  if (!bx.ensure(vb * 2 * nrhs) || (!on_device && !stage.ensure(vb * 2 * nrhs))) {
    h->st = keep;
    return MG_ENOMEM;
  }
  KSys full;
  full.n = n;
  full.apply = [&](const void* in, void* out) { return op_apply(h, 0, MG_F64, in, out, nullptr, 1.0, 0.0, nullptr, 0, 1); };
  full.resid = [&](const void* xx, void* r, const void* bb) {
    return op_apply(h, 0, MG_F64, xx, r, bb, -1.0, 1.0, nullptr, 0, 1);
  };
  auto body = [&]() -> int {
    RET(ensure_reducer(h, 1));
    const void* bs = b_ext;
    const void* xs = x_ext;
    if (!on_device) {
      CK(cudaMemcpyAsync(stage.p, b_ext, vb * nrhs, cudaMemcpyHostToDevice, h->st));
      CK(cudaMemcpyAsync((char*)stage.p + vb * nrhs, x_ext, vb * nrhs, cudaMemcpyHostToDevice, h->st));
      bs = stage.p;
      xs = (char*)stage.p + vb * nrhs;
    }
    double2* B = bx.as<double2>();
    double2* X = B + n * nrhs;
    LK(launch_ext_to_int(MG_F64, 12, 4, f.V, nrhs, bs, B, h->st));
    LK(launch_ext_to_int(MG_F64, 12, 4, f.V, nrhs, xs, X, h->st));
    int worst = MG_OK;
    for (int r = 0; r < nrhs; ++r) {
      auto t0 = std::chrono::steady_clock::now();
      mg_stats* sr = stats ? stats + r : nullptr;
      const int s = eo ? krylov_eo_one(h, base, B + n * r, X + n * r, tol, max_iter, sr)
                       : krylov_one(h, full, base, B + n * r, X + n * r, tol, max_iter, sr);
      if (s != MG_OK && s != MG_ENOCONV) return s;
      if (s == MG_ENOCONV) worst = s;
      if (stats) stats[r].solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    void* dst = on_device ? (void*)x_ext : stage.p;
    LK(launch_int_to_ext(MG_F64, 12, 4, f.V, nrhs, X, dst, h->st));
    if (!on_device) CK(cudaMemcpyAsync(x_ext, stage.p, vb * nrhs, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return worst;
  };
  rc = body();
  h->st = keep;
  return rc;
}

extern "C" int mg_solve(mg_handle* h, const double* b, double* x, int nrhs, int on_device, double tol,
                        mg_stats* stats, void* stream) {
  if (!h || !b || !x || nrhs < 1 || !(tol > 0.0)) {
    set_error("mg_solve: bad argument");
    return MG_EINVAL;
  }
  cudaStream_t keep = h->st;
  h->st = (cudaStream_t)stream;
  int rc = gcr_solve(h, b, x, nrhs, on_device, tol, stats);
  h->st = keep;
  return rc;
}

// Independent solves on one GPU at once: one host thread per handle, each on
// its own stream, so that the small launches of latency-bound solves (small
// lattices, few right-hand sides) from different handles fill the SMs
// together.  The first failing handle's status and message are returned.
// One multi-right-hand-side solve in which right-hand side r has its own mass
// m_r: D(m) = D(0) + m 1 and P^+ P = 1 (Eq. 2.3), so every level's operator
// at m_r is the handle's plus (m_r - mass) on the diagonal, applied per
// right-hand side inside the stencil kernels; the coarsest solve takes the
// inverse of its own mass.  The null vectors (built at the handle's mass)
// serve every mass, as for mg_retarget.
extern "C" int mg_solve_masses(mg_handle* h, const double* masses, const double* b, double* x, int nrhs, int on_device,
                               double tol, mg_stats* stats, void* stream) {
  if (!h || !masses || !b || !x || nrhs < 1 || nrhs > kMaxRhs || !(tol > 0.0)) {
    set_error("mg_solve_masses: bad argument");
    return MG_EINVAL;
  }
  if (h->p.fine_smoother != 0) {
    set_error("mg_solve_masses: a mass per right-hand side needs the MR fine smoother (fine_smoother = 0)");
    return MG_EINVAL;
  }
  std::vector<double> ms;
  std::vector<int> idx(kMaxRhs, 0);
  std::vector<double> adiag(kMaxRhs, 4.0 + h->mass), shift(kMaxRhs, 0.0);
  for (int r = 0; r < nrhs; ++r) {
    if (!isfinite(masses[r])) {
      set_error("mg_solve_masses: mass is not finite");
      return MG_EINVAL;
    }
    int z = 0;
    while (z < (int)ms.size() && ms[z] != masses[r]) ++z;
    if (z == (int)ms.size()) ms.push_back(masses[r]);
    idx[r] = z;
    adiag[r] = 4.0 + masses[r];
    shift[r] = masses[r] - h->mass;
  }
  cudaStream_t keep = h->st;
  h->st = (cudaStream_t)stream;
  auto body = [&]() -> int {
    if (!h->mm_adiag.ensure(kMaxRhs * sizeof(double)) || !h->mm_shift.ensure(kMaxRhs * sizeof(double)) ||
        !h->mm_idx.ensure(kMaxRhs * sizeof(int)))
      return MG_ENOMEM;
    if (h->lev.size() >= 2 && ms != h->mm_masses) RET(build_mass_inverses(h, ms));
    CK(cudaMemcpyAsync(h->mm_adiag.p, adiag.data(), kMaxRhs * sizeof(double), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->mm_shift.p, shift.data(), kMaxRhs * sizeof(double), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->mm_idx.p, idx.data(), kMaxRhs * sizeof(int), cudaMemcpyHostToDevice, h->st));
    h->mm_active = true;
    const int rc = gcr_solve(h, b, x, nrhs, on_device, tol, stats);
    h->mm_active = false;
    return rc;
  };
  const int rc = body();
  h->mm_active = false;
  h->st = keep;
  return rc;
}

extern "C" int mg_solve_many(mg_handle* const* hs, int count, const double* const* b, double* const* x, int nrhs,
                             int on_device, double tol, mg_stats* stats, void* const* streams) {
  if (!hs || !b || !x || count < 1 || nrhs < 1 || !(tol > 0.0)) {
    set_error("mg_solve_many: bad argument");
    return MG_EINVAL;
  }
  for (int i = 0; i < count; ++i) {
    bool bad = !hs[i] || !b[i] || !x[i];
    for (int j = 0; j < i; ++j) bad |= hs[i] == hs[j];
    if (bad) {
      set_error("mg_solve_many: handles must be distinct and non-null (a handle is not thread-safe), b and x "
                "non-null");
      return MG_EINVAL;
    }
  }
  std::vector<int> rc(count, MG_OK);
  std::vector<std::string> msg(count);
  auto run = [&](int i) {
    cudaStream_t st = streams ? (cudaStream_t)streams[i] : nullptr;
    bool own = false;
    if (!st) {
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        rc[i] = MG_ECUDA;
        msg[i] = "mg_solve_many: stream creation failed";
        return;
      }
      own = true;
    }
    rc[i] = mg_solve(hs[i], b[i], x[i], nrhs, on_device, tol, stats ? stats + (size_t)i * nrhs : nullptr, st);
    if (rc[i] != MG_OK) msg[i] = mg_last_error();
    if (own) cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  pool.reserve(count - 1);
  int started = 1;
  for (; started < count; ++started) {
    try {
      pool.emplace_back(run, started);
    } catch (const std::exception&) {  // no thread to be had: the rest run on this one
      break;
    }
  }
  run(0);
  for (int i = started; i < count; ++i) run(i);
  for (auto& t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (rc[i] != MG_OK) {
      set_error("handle " + std::to_string(i) + ": " + msg[i]);
      return rc[i];
    }
  return MG_OK;
}
