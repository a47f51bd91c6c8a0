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
  using Store = typename Prec<MODE>::Store;
  using Rest = typename Prec<MODE>::Rest;
  cudaStream_t s = c->stream;
  Geo G;
  G.nx = c->nx;
  G.ny = c->ny;
  G.nz = c->nz;
  G.wall = c->p.wall_last;
  G.N = c->N;
  G.P = c->P;
  G.P32 = (int)c->P;
  double* part = scratch;
  double* meas = scratch + 3 * TLB_STATIC_BLOCKS;
  // every partial slot, total and measure is overwritten below; nothing in
  // the scratch needs to start at zero
  k_mass_partials<L, MODE><<<TLB_STATIC_BLOCKS, 256, 0, s>>>(G, c->ptr<Store>(c->L.lo[c->cur]),
                                                             c->ptr<Rest>(c->L.rest[c->cur]), part);
  TLB_LAUNCHED(c, "k_mass_partials");
  k_reduce_partials<<<1, 256, 0, s>>>(part, TLB_STATIC_BLOCKS, 3, meas);
  TLB_LAUNCHED(c, "k_reduce_partials");
  if (c->ne > 0) {
    k_capsule_measures<<<c->ncap, 256, 0, s>>>(c->ptr<double>(c->L.X), c->ptr<int>(c->L.E), c->ptr<int>(c->L.ecap),
                                               c->ne, c->NV, c->ncap, meas + 4);
    TLB_LAUNCHED(c, "k_capsule_measures");
  }
  double h[4 + 2 * TLB_STATIC_MAX_CAPS];
  TLB_CUDA(cudaMemcpyAsync(h, meas, sizeof(h), cudaMemcpyDeviceToHost, s));
  unsigned st = 0;
  TLB_CUDA(cudaMemcpyAsync(&st, c->ptr<unsigned>(c->L.status), sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  TLB_CUDA(cudaStreamSynchronize(s));
  out->step = c->t;
  for (int q = 0; q < 3; ++q) out->mass[q] = h[q];
  out->umax = 0;
  out->n_caps = c->ncap;
  for (int k = 0; k < 8; ++k) {
    out->area[k] = k < c->ncap ? h[4 + 2 * k] : 0;
    out->volume[k] = k < c->ncap ? h[4 + 2 * k + 1] : 0;
  }
  if (st & ST_NAN) { set_error("diagnostics: NaN in the populations"); return TLB_ERR_DIVERGED; }
  if (st & ST_MARKER_JUMP) { set_error("diagnostics: a marker moved half a cell in one step"); return TLB_ERR_DIVERGED; }
  if (st & ST_OVERFLOW) { set_error("diagnostics: spreading bin overflow"); return TLB_ERR_DIVERGED; }
  return TLB_OK;
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
