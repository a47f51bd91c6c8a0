// tlb_diagnostics_static: the FP64 diagnostics of tlb_diagnostics computed
// with reduction scratch held in a fixed device array of this file instead
// of the caller's arena.  It exists for callers that cannot provide device
// memory at the point of the call -- for example code that runs inside a
// frame or a real-time loop where cudaMalloc (which synchronises the device)
// is not allowed, or whose device memory is owned by another runtime -- and
// that cannot spare the arena's scratch region because another stream is
// using it.  The call allocates nothing.
#include <mutex>

#include "tlb_ctx.h"
#include "tlb_ibm.cuh"
#include "tlb_lb.cuh"
#include "tlb_diag.cuh"

// Partial sums of up to TLB_STATIC_BLOCKS reduction blocks for the three
// totals, then the totals themselves and two measures per capsule.  Every
// GPU that loads the library holds this array (about 26 KB) until exit.
#define TLB_STATIC_BLOCKS 1024
#define TLB_STATIC_MAX_CAPS 8
#define TLB_STATIC_DOUBLES (3 * TLB_STATIC_BLOCKS + 4 + 2 * TLB_STATIC_MAX_CAPS)
static __device__ __align__(256) double g_diag_scratch[TLB_STATIC_DOUBLES];

// Device address of g_diag_scratch on the device that holds the context's
// arena, looked up once per device with that device current (the host-side
// symbol is not a device address); the caller's current device is restored.
static std::mutex g_scratch_mu;
static double* g_scratch_addr[64] = {nullptr};

static tlb_status scratch_address(const Ctx* c, double** out) {
  cudaPointerAttributes at;
  TLB_CUDA(cudaPointerGetAttributes(&at, c->base));
  const int dev = at.device;
  if (dev < 0 || dev >= 64) {
    set_error("tlb_diagnostics_static: the arena is not on a device with ordinal 0..63");
    return TLB_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    int prev = 0;
    TLB_CUDA(cudaGetDevice(&prev));
    if (prev != dev) TLB_CUDA(cudaSetDevice(dev));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_diag_scratch);
    if (prev != dev) TLB_CUDA(cudaSetDevice(prev));
    if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(g_diag_scratch)");
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return TLB_OK;
}

template <class L, int MODE>
static tlb_status run_static(Ctx* c, double* scratch, tlb_diag* out) {
  return fp64_diagnostics<L, MODE>(c, scratch, TLB_STATIC_BLOCKS, scratch + 3 * TLB_STATIC_BLOCKS, out);
}

extern "C" tlb_status tlb_diagnostics_static(void* ctx, tlb_diag* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !out) { set_error("ctx/out is NULL"); return TLB_ERR_ARG; }
  if (c->ncap > TLB_STATIC_MAX_CAPS) {
    set_error("tlb_diagnostics_static: at most 8 capsules fit the static scratch");
    return TLB_ERR_ARG;
  }
  double* scratch = nullptr;
  tlb_status st = scratch_address(c, &scratch);
  if (st != TLB_OK) return st;
  // moment storage: the populations the moments stand for (no allocation)
  if ((st = c->impl->sync_pops(c)) != TLB_OK) return st;
  switch (c->p.dim * 10 + c->p.storage) {
    case 20: return run_static<D2Q9, TLB_F64>(c, scratch, out);
    case 21: return run_static<D2Q9, TLB_F32>(c, scratch, out);
    case 31: return run_static<D3Q19, TLB_F32>(c, scratch, out);
    case 32: return run_static<D3Q19, TLB_F16>(c, scratch, out);
    case 33: return run_static<D3Q19, TLB_BF16>(c, scratch, out);
    default: set_error("tlb_diagnostics_static: unsupported dim/storage"); return TLB_ERR_ARG;
  }
}
