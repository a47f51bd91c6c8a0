// FP64 diagnostics of a context (tlb_diagnostics, tlb_diagnostics_static):
// the population totals (fixed-order block partials, then one reduction
// block), the capsule areas and volumes, and the status word decoded into
// the call's error.  The reduction scratch is the caller's: the arena's
// region or the static array of tlb_static.cu.
#pragma once
#include "tlb_ctx.h"
#include "tlb_ibm.cuh"
#include "tlb_lb.cuh"

// part: nb * 3 doubles; meas: 4 + 2 * ncap doubles (at most 8 capsules read
// back); the populations must be current (sync_pops).
template <class L, int MODE>
tlb_status fp64_diagnostics(Ctx* c, double* part, int nb, double* meas, tlb_diag* out) {
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
  // every partial slot, total and measure is overwritten below
  k_mass_partials<L, MODE><<<nb, 256, 0, s>>>(G, c->ptr<Store>(c->L.lo[c->cur]), c->ptr<Rest>(c->L.rest[c->cur]),
                                              part);
  TLB_LAUNCHED(c, "k_mass_partials");
  k_reduce_partials<<<1, 256, 0, s>>>(part, nb, 3, meas);
  TLB_LAUNCHED(c, "k_reduce_partials");
  if (c->ne > 0) {
    k_capsule_measures<<<c->ncap, 256, 0, s>>>(c->ptr<double>(c->L.X), c->ptr<int>(c->L.E), c->ptr<int>(c->L.ecap),
                                               c->ne, c->NV, c->ncap, meas + 4);
    TLB_LAUNCHED(c, "k_capsule_measures");
  }
  double h[4 + 16];
  const int nread = 4 + 2 * (c->ncap < 8 ? c->ncap : 8);
  TLB_CUDA(cudaMemcpyAsync(h, meas, nread * sizeof(double), cudaMemcpyDeviceToHost, s));
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
