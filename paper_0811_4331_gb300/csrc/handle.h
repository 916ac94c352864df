// Internal state of an mg_handle and device-memory helpers (host code).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <shared_mutex>
#include <string>
#include <vector>

#include "../../include/wilson_mg.h"
#include "kernels.h"

namespace wmg {

void set_error(const std::string& msg);

// Graph captures hold this shared; a device-wide synchronisation (which would
// invalidate a capture running on another thread) needs it exclusively and is
// skipped when it cannot have it at once.
inline std::shared_mutex g_capture_mu;

// Device buffers the library has taken since it was loaded, from the driver
// or from its cache of freed buffers (a monotonic count).
inline std::atomic<unsigned long long> g_dev_allocs{0};

// Cache of device memory.  A buffer the library frees goes back to a
// process-wide list keyed by its size class, and the next buffer of that
// class is taken from the list instead of from cudaMalloc: a solve that
// builds and destroys hierarchies (the mass sweep builds five per step) then
// allocates from the driver only the first time.  A block enters the list
// only when no GPU work can still use it: release() synchronises the device
// first (what cudaFree does implicitly) and, if that synchronisation fails,
// holds the block back until a later one succeeds; inside a DevIdleScope,
// whose creator has synchronised, blocks go back at once (mg_destroy, and
// temporaries whose stream was synchronised).  mg_trim_cache hands the
// cached blocks back to the driver.
struct DevCache {
  std::mutex mu;
  std::map<size_t, std::vector<void*>> blocks;
  // blocks released when a device synchronisation failed (e.g. while another thread was capturing a
  // graph): they join `blocks` after the next successful one
  std::vector<std::pair<void*, size_t>> pending;
  // size classes: powers of two up to 4 KiB, then eight steps per octave (at most 1/8 unused)
  static size_t size_class(size_t n) {
    if (n <= 4096) {
      size_t c = 256;
      while (c < n) c <<= 1;
      return c;
    }
    size_t k = 4096;
    while (k * 2 <= n) k <<= 1;
    const size_t step = k / 8;
    return (n + step - 1) / step * step;
  }
  void* take(size_t c) {
    std::lock_guard<std::mutex> lk(mu);
    auto it = blocks.find(c);
    if (it == blocks.end() || it->second.empty()) return nullptr;
    void* p = it->second.back();
    it->second.pop_back();
    return p;
  }
  void give(void* p, size_t c) {
    std::lock_guard<std::mutex> lk(mu);
    blocks[c].push_back(p);
  }
  // A block that work still queued on any stream may use: reusable once the device has synchronised.
  void give_after_sync(void* p, size_t c) {
    bool synced = false;
    {
      std::unique_lock<std::shared_mutex> nocapture(g_capture_mu, std::try_to_lock);
      if (nocapture.owns_lock()) synced = cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!synced) cudaGetLastError();  // leave no error behind for this thread's next launch check
    std::lock_guard<std::mutex> lk(mu);
    if (synced) {
      for (auto& q : pending) blocks[q.second].push_back(q.first);
      pending.clear();
      blocks[c].push_back(p);
    } else {
      pending.push_back({p, c});
    }
  }
  // Free every cached block (after a device synchronisation); returns the bytes freed.
  size_t trim() {
    std::unique_lock<std::shared_mutex> nocapture(g_capture_mu);
    const bool synced = cudaDeviceSynchronize() == cudaSuccess;
    if (!synced) cudaGetLastError();
    std::lock_guard<std::mutex> lk(mu);
    size_t freed = 0;
    for (auto& kv : blocks) {
      for (void* p : kv.second) cudaFree(p);
      freed += kv.first * kv.second.size();
    }
    blocks.clear();
    if (synced) {
      for (auto& q : pending) {
        cudaFree(q.first);
        freed += q.second;
      }
      pending.clear();
    }
    return freed;
  }
};
inline DevCache& dev_cache() {
  static DevCache* c = new DevCache();  // never destroyed: buffers may be released at process exit
  return *c;
}
inline thread_local bool tl_dev_idle = false;
// While alive, buffers released on this thread skip the device synchronisation.
struct DevIdleScope {
  bool prev;
  DevIdleScope() : prev(tl_dev_idle) { tl_dev_idle = true; }
  ~DevIdleScope() { tl_dev_idle = prev; }
};

// Owning device buffer (capacity `bytes`, a size class of DevCache).  Nothing
// is shared between handles.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      if (tl_dev_idle)
        dev_cache().give(p, bytes);
      else
        dev_cache().give_after_sync(p, bytes);
    }
    p = nullptr;
    bytes = 0;
  }
  // Release after the caller has synchronised every stream that used the buffer.
  void release_idle() {
    if (p) dev_cache().give(p, bytes);
    p = nullptr;
    bytes = 0;
  }
  // (Re)allocate to at least n bytes; returns false on failure.
  bool ensure(size_t n) {
    if (n <= bytes && p) return true;
    release();
    if (n == 0) n = 16;
    const size_t c = DevCache::size_class(n);
    p = dev_cache().take(c);
    if (!p && cudaMalloc(&p, c) != cudaSuccess) {
      cudaGetLastError();
      dev_cache().trim();  // retry once with the cached blocks handed back
      if (cudaMalloc(&p, c) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return false;
      }
    }
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    bytes = c;
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
