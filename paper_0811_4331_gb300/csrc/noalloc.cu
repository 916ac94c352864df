// MR smoothing without any device allocation, for callers that cannot
// allocate device memory at the time of the call.
//
// mr_apply needs scratch beyond its inputs and outputs: the work vector
// p = A r and the grid-reduction partial sums, ticket counter and result
// slot behind the deterministic dot products.  mr_apply takes that scratch
// from buffers the handle allocates on demand with cudaMalloc.  Some callers
// cannot allow that at call time: code running inside a pre-allocated
// memory budget (a serving process that fixed its footprint at start-up), a
// host thread that must not take the driver's allocation locks while other
// streams run, or a framework that forbids allocation inside its own step.
// mr_apply_noalloc runs the same kernels with the same launch shapes but
// takes all scratch from one file-scope __device__ array of fixed size.
#include <mutex>
#include <string>

#include "handle.h"

namespace {

// Fixed scratch: 16 MiB in every GPU that loads this library, held until exit.
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code g_noalloc_scratch names a host-side stand-in, not the device
// array; the device address is looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    wmg::set_error(std::string("mr_apply_noalloc: cudaGetDevice failed: ") + cudaGetErrorString(e));
    return MG_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      wmg::set_error(std::string("mr_apply_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return MG_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MG_OK;
}

inline size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }
inline size_t elem_bytes(int prec) { return prec == MG_F64 ? 16 : (prec == MG_F32 ? 8 : 4); }

}  // namespace

using namespace wmg;

// A coarse level in FP32 with the tensor-core stencil runs on it, as in mr_apply.
static bool uses_mma(const Level& a, int l, int prec) { return l > 0 && a.cop_mma.p && prec == MG_F32; }

// out = a_ A_l in + c_ y, optional dots into `red` (the kernels mr_apply runs).
static int apply_level(mg_handle* h, int l, int prec, const void* in, void* out, const void* y, double a_,
                       double c_, const void* z, const RedArgs& red, cudaStream_t st) {
  Level& a = *h->lev[l];
  int rc;
  if (uses_mma(a, l, prec)) {
    // tensor cores: out = a_ A in + c_ y, then the dots in a separate deterministic pass
    rc = launch_coarse_mma(prec, a.cop_mma.p, in, out, y, a.L, a.ncomp, 1, a_, c_, st);
    if (rc == 0 && z) rc = launch_dot(prec, a.n(), 1, out, z, red, st);
  } else if (l == 0) {
    DslashCall d;
    d.prec = prec;
    d.in = in;
    d.out = out;
    d.y = y;
    d.z = z;
    d.links = a.links[prec].p;
    for (int m = 0; m < 4; ++m) d.L[m] = a.L[m];
    d.a = a_ * (4.0 + h->mass);
    d.b = -0.5 * a_;
    d.c = c_;
    d.nrhs = 1;
    d.red = red;
    rc = launch_wilson(d, st);
  } else {
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
    k.nrhs = 1;
    k.red = red;
    rc = launch_coarse_apply(k, st);
  }
  return rc == 0 ? MG_OK : MG_ECUDA;
}

extern "C" int mr_apply_noalloc(mg_handle* h, int level, int prec, const void* b, void* x, void* r, int steps,
                                void* stream) {
  if (!h || level < 0 || level >= (int)h->lev.size() || !b || !x || !r || steps < 0 || prec < 0 || prec > 3) {
    set_error("mr_apply_noalloc: bad argument");
    return MG_EINVAL;
  }
  Level& a = *h->lev[level];
  const bool mma = uses_mma(a, level, prec);
  if ((level == 0 && !a.links[prec].p) || (level > 0 && !mma && !a.cop[prec].p)) {
    set_error("mr_apply_noalloc: operator not stored in this precision");
    return MG_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // carve the fixed scratch: p | partial sums | tickets | result slot
  const size_t n = a.n();
  const size_t partials = mma ? (size_t)red_blocks(n) * 4
                               : (level == 0 ? (size_t)wilson_blocks(a.V) : (size_t)coarse_blocks(a.ncomp, a.V)) * 3;
  const size_t off_part = align256(n * elem_bytes(prec));
  const size_t off_tick = off_part + align256(partials * sizeof(double));
  const size_t off_slot = off_tick + 256;
  const size_t need = off_slot + 256;
  if (need > kNoAllocScratchBytes) {
    set_error("mr_apply_noalloc: level needs " + std::to_string(need) + " bytes of scratch; the fixed scratch holds " +
              std::to_string(kNoAllocScratchBytes));
    return MG_EINVAL;
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != MG_OK) return rc;
  char* s = (char*)base;
  void* p = s;
  RedArgs red;
  red.partials = (double*)(s + off_part);
  red.tickets = (unsigned*)(s + off_tick);
  red.result = (double*)(s + off_slot);
  red.stride = 4;
  // tickets must start at zero; the slot is written before it is read
  cudaError_t e = cudaMemsetAsync(red.tickets, 0, 256, st);
  if (e != cudaSuccess) {
    set_error(std::string("mr_apply_noalloc: ") + cudaGetErrorString(e));
    return MG_ECUDA;
  }
  // r = b - A x, then `steps` under-relaxed MR steps
  rc = apply_level(h, level, prec, x, r, b, -1.0, 1.0, nullptr, red, st);
  for (int k = 0; k < steps && rc == MG_OK; ++k) {
    rc = apply_level(h, level, prec, r, p, nullptr, 1.0, 0.0, r, red, st);
    if (rc != MG_OK) break;
    MrUpdate m;
    m.prec = prec;
    m.n = n;
    m.nrhs = 1;
    m.x_out = x;
    m.x_in = x;
    m.u = r;
    m.r_out = r;
    m.r_in = r;
    m.p = p;
    m.dots = red.result;
    m.dstride = 4;
    m.omega = h->p.omega;
    m.red = red;
    m.red.result = nullptr;
    rc = launch_mr_update(m, st) == 0 ? MG_OK : MG_ECUDA;
  }
  if (rc != MG_OK) {
    cudaError_t le = cudaGetLastError();
    set_error(std::string("mr_apply_noalloc: launch failed: ") + cudaGetErrorString(le));
  }
  return rc;
}
