// Internal state of an mg_handle and device-memory helpers (host code).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <memory>
#include <string>
#include <vector>

#include "../../include/wilson_mg.h"
#include "kernels.h"

namespace wmg {

void set_error(const std::string& msg);

// Device allocations the library has made since it was loaded (successful cudaMalloc calls).
inline std::atomic<unsigned long long> g_dev_allocs{0};

// Owning device buffer.  The library allocates with cudaMalloc and frees on
// destruction; nothing is shared between handles.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // (Re)allocate to at least n bytes; returns false on failure.
  bool ensure(size_t n) {
    if (n <= bytes && p) return true;
    release();
    if (n == 0) n = 16;
    if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    bytes = n;
    return true;
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

struct Level {
  int L[4] = {0, 0, 0, 0};
  int V = 0;
  int ncomp = 0;  // 12 on level 0, 2 nv_{l-1} on level l >= 1
  int q = 1;      // chunk of the level's fields: 4 on level 0 (chunked layout), 1 on coarse levels
  // coarsening to level l+1 (nv == 0 on the coarsest level)
  int nv = 0;
  int blk[4] = {1, 1, 1, 1};
  int bsites = 0;  // sites per aggregate
  int nhalf = 0;   // components per chirality = ncomp / 2
  int Lc[4] = {0, 0, 0, 0};
  int Vc = 0;
  int sweeps = 0;
  int cycles = 1;
  // operator of this level, per storage precision (index = precision code)
  DevBuf links[4];  // level 0: 4 V NL complex in the link layout of wilson_hop.cuh
  DevBuf links_eo[4];  // level 0, even-odd kernels: the same with the sites parity-major (built on first use)
  DevBuf cop[4];    // level >= 1: stencil [9][ncomp][ncomp][V]
  DevBuf cop_mma;   // level >= 1 (coarse_mma): BF16 stencil in MMA fragment order
  // prolongator to level l+1, per precision: [Vc][2][nv][nhalf][bsites]
  DevBuf P[4];
  // coarsest level: dense inverse [N][N], N = ncomp V, FP64 (plain) or FP32
  // (mixed: applied with FP64 iterative refinement)
  DevBuf inv;
  DevBuf mm_scratch;  // partial tiles and tickets of the many-right-hand-side inverse product
  int inv_prec = 0;
  bool inv_pending = false;  // coarsest inverse deferred (mg_params.defer_coarsest), built on first use
  int N() const { return ncomp * V; }
  size_t n() const { return (size_t)ncomp * V; }
};

struct Reducer {
  DevBuf partials, tickets, slots;
  size_t max_partials = 0;  // doubles
  int nslots = 0;
  bool init(size_t partial_doubles, int slots_doubles, int ntickets) {
    if (!partials.ensure(partial_doubles * sizeof(double))) return false;
    if (!tickets.ensure((size_t)ntickets * sizeof(unsigned))) return false;
    if (!slots.ensure((size_t)slots_doubles * sizeof(double))) return false;
    if (cudaMemset(tickets.p, 0, (size_t)ntickets * sizeof(unsigned)) != cudaSuccess) return false;
    if (cudaMemset(slots.p, 0, (size_t)slots_doubles * sizeof(double)) != cudaSuccess) return false;
    max_partials = partial_doubles;
    nslots = slots_doubles;
    return true;
  }
  // Reduction descriptor writing into result slot `slot` (doubles offset).
  RedArgs at(size_t slot, int stride) const {
    RedArgs r;
    r.partials = partials.as<double>();
    r.tickets = tickets.as<unsigned>();
    r.result = slots.as<double>() + slot;
    r.stride = stride;
    return r;
  }
  double* slot(size_t off) const { return slots.as<double>() + off; }
};

}  // namespace wmg

struct mg_handle {
  mg_params p;
  double mass = 0.0;
  int dims[4] = {0, 0, 0, 0};
  cudaStream_t st = nullptr;
  std::vector<std::unique_ptr<wmg::Level>> lev;
  wmg::Reducer red;
  // work vectors: [level][precision][index]
  std::vector<std::vector<std::vector<std::unique_ptr<wmg::DevBuf>>>> work;
  int work_nrhs = 0;
  // outer solver buffers
  wmg::DevBuf gr, gW, gZ, gb64, gx64, gr64, gtmp;
  wmg::DevBuf gH, galpha, gy;  // outer GCR: H (A Z = W H), alpha, y = H^-1 alpha per right-hand side
  wmg::DevBuf err_flag;  // device int set by setup kernels on failure
  // profiler: event pairs per (class, precision)
  unsigned prof_mask = 0;
  std::vector<cudaEvent_t> prof_pool;
  size_t prof_used = 0;
  struct ProfMark {
    int key;       // class * 4 + prec
    size_t idx;    // index of the start event
    double bytes;  // algorithmic bytes of the interval (0: not counted)
  };
  std::vector<ProfMark> prof_marks;
  // CUDA graphs of the V-cycle, keyed by (nrhs, input, output, buffer generation)
  struct CycleGraph {
    bool mm;  // captured with a mass per right-hand side
    int nrhs;
    const void* in;
    void* out;
    unsigned long long gen;
    unsigned long long nodes;
    cudaGraphExec_t exec;
  };
  std::vector<CycleGraph> graphs;
  // solves with a mass per right-hand side (mg_solve_masses): per right-hand side 4 + m_r and m_r - mass
  // (FP64, kMaxRhs each), the index of its coarsest inverse, and the inverses [count][N][N] of the
  // distinct masses in mm_masses
  bool mm_active = false;
  wmg::DevBuf mm_adiag, mm_shift, mm_idx, mm_inv;
  std::vector<double> mm_masses;
  unsigned long long buf_gen = 1;  // bumped whenever a work buffer or the reducer is reallocated
  cudaStream_t cap_st = nullptr;   // private stream used only for capture
  bool capturing = false;
  bool use_graphs = true;
  double* host_slots = nullptr;  // pinned mirror for read-backs
};
