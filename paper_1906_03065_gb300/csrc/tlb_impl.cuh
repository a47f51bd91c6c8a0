// Templated host driver: builds kernel arguments from the context and
// enqueues the step of the method on the context stream.
#pragma once
#include <math.h>

#include <vector>

#include "tlb_ctx.h"
#include "tlb_ibm.cuh"
#include "tlb_lb.cuh"
#include "tlb_measure.cuh"
#include "tlb_diag.cuh"

template <class L, int MODE>
struct Impl : ImplBase {
  using Real = typename Prec<MODE>::Real;
  using Store = typename Prec<MODE>::Store;
  using Rest = typename Prec<MODE>::Rest;

  static Geo geo(const Ctx* c) {
    Geo g;
    g.nx = c->nx;
    g.ny = c->ny;
    g.nz = c->nz;
    g.wall = c->p.wall_last;
    g.N = c->N;
    g.P = c->P;
    g.P32 = (int)c->P;
    return g;
  }

  static LBArgs<MODE> lbargs(Ctx* c, int src) {
    LBArgs<MODE> a;
    a.G = geo(c);
    a.lo_src = c->ptr<Store>(c->L.lo[src]);
    a.rest_src = c->ptr<Rest>(c->L.rest[src]);
    a.lo_dst = c->ptr<Store>(c->L.lo[1 - src]);
    a.rest_dst = c->ptr<Rest>(c->L.rest[1 - src]);
    a.rho = c->ptr<Real>(c->L.rho);
    a.phi = c->ptr<Real>(c->L.phi);
    a.psi = c->ptr<Real>(c->L.psi);
    // rho - 1 and j for the tau = 1 collide (the moments write them only then)
    a.jm = variant_t1(c->tile_variant) ? c->ptr<Real>(c->L.jm) : nullptr;
    // moment storage: the collide stores the moments, the pull rebuilds from them
    a.mst = c->moments() ? c->ptr<Real>(c->L.M) : nullptr;
    a.msrc = a.mst;
    a.I = c->ptr<Real>(c->L.I);
    a.fib = c->ptr<Real>(c->L.fib);
    a.ftot = c->ptr<Real>(c->L.ftot);
    a.bflag = c->ptr<unsigned char>(c->L.bflag);
    a.nbx = c->nbx;
    a.nby = c->nby;
    a.fe.k1 = (Real)c->p.kappa[0];
    a.fe.k2 = (Real)c->p.kappa[1];
    a.fe.k3 = (Real)c->p.kappa[2];
    a.fe.kc = (Real)c->p.kappa_c;
    a.fe.a2 = (Real)(c->p.alpha * c->p.alpha);
    a.om = (Real)(1.0 / c->p.tau);
    a.om_phi = (Real)(1.0 / c->p.tau_phi);
    a.om_psi = (Real)(1.0 / c->p.tau_psi);
    a.gphi = (Real)c->p.gamma_phi;
    a.gpsi = (Real)c->p.gamma_psi;
    a.zc = c->tiles_zc;
    a.forcing = c->p.forcing;
    a.status = c->ptr<unsigned>(c->L.status);
    return a;
  }

  static IBArgs<Real> ibargs(Ctx* c) {
    IBArgs<Real> a;
    a.G = geo(c);
    a.dim = c->p.dim;
    a.NV = c->NV;
    a.nn = c->nn;
    a.ne = c->ne;
    a.X = c->ptr<double>(c->L.X);
    a.E = c->ptr<int>(c->L.E);
    a.ecap = c->ptr<int>(c->L.ecap);
    a.ncap = c->ptr<int>(c->L.ncap);
    const double* cp = c->ptr<double>(c->L.cap_par);
    a.ks = cp;
    a.kb = cp + c->ncap;
    a.sG = cp + 2 * c->ncap;
    a.sC = cp + 3 * c->ncap;
    a.ds0 = c->ptr<double>(c->L.ds0);
    a.rprev = c->ptr<int>(c->L.rprev);
    a.rnext = c->ptr<int>(c->L.rnext);
    a.A0 = c->ptr<double>(c->L.A0);
    a.G0i = c->ptr<double>(c->L.G0i);
    a.inc_off = c->ptr<int>(c->L.inc_off);
    a.inc = c->ptr<int>(c->L.inc);
    a.adj = c->ptr<int>(c->L.adj);
    a.ring_off = c->ptr<int>(c->L.ring_off);
    a.ring = c->ptr<int>(c->L.ring);
    a.nedge = c->nedge;
    a.edges = c->ptr<int>(c->L.edges);
    a.en = c->ptr<Real>(c->L.en);
    a.vn = c->ptr<Real>(c->L.vn);
    a.erel = c->ptr<Real>(c->L.erel);
    a.eorg = c->ptr<int>(c->L.eorg);
    a.ecst = c->ptr<Real>(c->L.ecst);
    a.xo = c->ptr<int>(c->L.xo);
    a.xr = c->ptr<Real>(c->L.xr);
    a.skc = c->ptr<Real>(c->L.skc);
    a.capr = c->ptr<Real>(c->L.capr);
    a.ncaps = c->ncap;
    a.ncpl = c->ptr<unsigned long long>(c->L.ncpl);
    a.F = c->ptr<Real>(c->L.F);
    a.box = c->ptr<int>(c->L.box);
    a.boxc = c->ptr<int>(c->L.box) + 6;
    a.key = c->ptr<unsigned long long>(c->L.key);
    a.own = c->ptr<int>(c->L.own);
    a.I = c->ptr<Real>(c->L.I);
    a.dsel = c->ptr<Real>(c->L.dsel);
    a.psi = c->ptr<Real>(c->L.psi);
    a.M = c->moments() ? c->ptr<Real>(c->L.M) : nullptr;
    a.fib = c->ptr<Real>(c->L.fib);
    a.ftot = c->ptr<Real>(c->L.ftot);
    a.bflag = c->ptr<unsigned char>(c->L.bflag);
    a.bcnt = c->ptr<int>(c->L.bcnt);
    a.bprev = c->ptr<int>(c->L.bprev);
    a.bcur = c->ptr<int>(c->L.bcur);
    a.boff = c->ptr<int>(c->L.boff);
    a.blist = c->ptr<int>(c->L.blist);
    a.bact = c->ptr<int>(c->L.bact);
    a.ctr = c->ptr<int>(c->L.ctr);
    a.nbx = c->nbx;
    a.nby = c->nby;
    a.nbz = c->nbz;
    a.nbricks = c->nbricks;
    a.alpha = (Real)c->p.alpha;
    a.dc = (Real)c->p.dc;
    a.kc = (Real)c->p.kappa_c;
    a.Iin = (Real)(0.5 * (1.0 + tanh(c->p.dc / (2.0 * c->p.alpha))));
    a.Iout = (Real)(0.5 * (1.0 + tanh(-c->p.dc / (2.0 * c->p.alpha))));
    a.status = c->ptr<unsigned>(c->L.status);
    return a;
  }

  static unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

  // Work of a step that depends on the marker positions X(t) only (element
  // and vertex normals and the distance scatter here; elastic forces and the
  // brick binning in ibm_bins).  It runs on the side stream while the
  // moments of the step are computed.
  // With snap the geometry kernel also takes the marker box's snapshot (the
  // advection's accumulator) and resets it.
  static tlb_status ibm_positions(Ctx* c, IBArgs<Real>& a, cudaStream_t s, bool snap = false) {
    k_geometry<Real><<<blocks((long long)c->ne + c->nn, 128), 128, 0, s>>>(a, snap ? 1 : 0);
    TLB_LAUNCHED(c, "k_geometry");
    const long long nfeat = (long long)c->ne + c->nedge + c->nn;
    constexpr int sw = scatter_warps<Real>();
    const unsigned nvb = SCAT_SPLIT * blocks(nfeat, 32 * sw);
    k_dist_scatter<Real><<<std::min(nvb, 4u * (unsigned)c->nsm), 32 * sw, 0, s>>>(a, (int)nvb);
    TLB_LAUNCHED(c, "k_dist_scatter");
    return TLB_OK;
  }

  // The step's marker box: recompute the accumulator if the markers were
  // overwritten, copy it to the snapshot every kernel of the step reads, and
  // reset it for the advection of this step.
  static tlb_status snapshot_box(Ctx* c, IBArgs<Real>& a, cudaStream_t s, bool fresh) {
    if (fresh) {
      TLB_CUDA(cudaMemsetAsync(a.box, 0x7F, 6 * sizeof(int), s));
      k_box<Real><<<blocks(c->nn, 128), 128, 0, s>>>(a);
      TLB_LAUNCHED(c, "k_box");
    }
    TLB_CUDA(cudaMemcpyAsync((void*)a.boxc, a.box, 6 * sizeof(int), cudaMemcpyDeviceToDevice, s));
    TLB_CUDA(cudaMemsetAsync(a.box, 0x7F, 6 * sizeof(int), s));
    return TLB_OK;
  }

  // Elastic forces and the binning of markers into spreading bricks (the
  // bins are consumed and reset by k_spread of the same step).
  static tlb_status ibm_bins(Ctx* c, IBArgs<Real>& a, cudaStream_t s) {
    k_node_forces<Real><<<blocks((long long)c->nn * 32, 128), 128, 0, s>>>(a);  // (clears ctr)
    TLB_LAUNCHED(c, "k_node_forces");
    k_brick_count<Real><<<blocks(c->nn, 128), 128, 0, s>>>(a);
    TLB_LAUNCHED(c, "k_brick_count");
    k_brick_compact<Real><<<blocks(c->nbricks, 256), 256, 0, s>>>(a);
    TLB_LAUNCHED(c, "k_brick_compact");
    k_brick_fill<Real><<<blocks(c->nn, 128), 128, 0, s>>>(a);
    TLB_LAUNCHED(c, "k_brick_fill");
    return TLB_OK;
  }

  // Profile I of the band and the coupling sums (needs psi(t)); the rest of
  // the box (column fill).
  static tlb_status launch_band(Ctx* c, IBArgs<Real>& a, cudaStream_t s) {
    k_band<Real><<<8 * c->nsm, 256, 0, s>>>(a);
    TLB_LAUNCHED(c, "k_band");
    return TLB_OK;
  }
  static tlb_status launch_fill(Ctx* c, IBArgs<Real>& a, cudaStream_t s) {
    k_fill<Real><<<blocks((long long)c->nx * c->ny * 32, 256), 256, 0, s>>>(a);
    TLB_LAUNCHED(c, "k_fill");
    return TLB_OK;
  }
  static tlb_status ibm_band(Ctx* c, IBArgs<Real>& a, cudaStream_t s) {
    tlb_status st = launch_band(c, a, s);
    return st == TLB_OK ? launch_fill(c, a, s) : st;
  }

  static tlb_status ibm_spread(Ctx* c, IBArgs<Real>& a, cudaStream_t s) {
    k_spread<Real><<<min(c->nbricks, 8 * c->nsm), 64, 0, s>>>(a);
    TLB_LAUNCHED(c, "k_spread");
    return TLB_OK;
  }

  tlb_status init_fields(Ctx* c, const double* C, const double* u) override {
    cudaStream_t s = c->stream;
    const long long N = c->N;
    IBArgs<Real> ia = ibargs(c);
    // membrane profile I(X0) (I_out everywhere when there are no membranes)
    if (c->nn > 0) {
      tlb_status st = snapshot_box(c, ia, s, true);
      if (st == TLB_OK) st = ibm_positions(c, ia, s);
      if (st == TLB_OK) st = ibm_band(c, ia, s);
      if (st != TLB_OK) return st;
      c->box_stale = true;  // the first step recomputes the box of X0
    }
    Real* rho = c->ptr<Real>(c->L.rho);
    Real* phi = c->ptr<Real>(c->L.phi);
    Real* psi = c->ptr<Real>(c->L.psi);
    Real* uf = c->ptr<Real>(c->L.ftot);  // velocity (free before the first step)
    // the caller's arrays go to the other population buffer (free until the
    // first step; at least 48 bytes per cell) and are converted on the device
    double* scratch = c->ptr<double>(c->L.lo[1 - c->cur]);
    const double* Cd = nullptr;
    const double* ud = nullptr;
    if (C) {
      TLB_CUDA(cudaMemcpyAsync(scratch, C, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s));
      Cd = scratch;
    }
    if (u) {
      TLB_CUDA(cudaMemcpyAsync(scratch + 3 * N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s));
      ud = scratch + 3 * N;
    }
    TLB_CUDA(cudaMemsetAsync(c->ptr<char>(c->L.ftot), 0, c->L.ftot.bytes, s));
    k_init_fields<Real><<<blocks(N, 256), 256, 0, s>>>(geo(c), c->p.dim, Cd, ud, c->p.u0[0], c->p.u0[1], c->p.u0[2],
                                                       c->p.alpha, c->p.interface_pos, c->ptr<Real>(c->L.I), rho,
                                                       phi, psi, uf);
    TLB_LAUNCHED(c, "k_init_fields");
    Geo G = geo(c);
    LBArgs<MODE> la = lbargs(c, c->cur);
    Real* mu = c->ptr<Real>(c->L.mu);
    k_mu_global<L, MODE><<<blocks(N, 256), 256, 0, s>>>(G, la.fe, rho, phi, psi, la.I, mu);
    TLB_LAUNCHED(c, "k_mu_global");
    k_init_eq<L, MODE><<<blocks(N, 256), 256, 0, s>>>(G, rho, phi, psi, uf, mu, la.gphi, la.gpsi,
                                                       c->ptr<Store>(c->L.lo[c->cur]),
                                                       c->ptr<Rest>(c->L.rest[c->cur]));
    TLB_LAUNCHED(c, "k_init_eq");
    TLB_CUDA(cudaMemsetAsync(c->ptr<char>(c->L.ftot), 0, c->L.ftot.bytes, s));
    // the initial state is the first reference of the equilibrium residual
    tlb_status rs = residual_launch(c);
    if (rs != TLB_OK) return rs;
    TLB_CUDA(cudaStreamSynchronize(s));
    c->t = 0;
    c->t_snap = 0;
    c->initialised = true;
    c->state_in_pops = true;  // (moment storage: the first step pulls these populations)
    c->pops_stale = false;
    return TLB_OK;
  }

  tlb_status sync_pops(Ctx* c) override {
    if (!c->moments() || c->state_in_pops || !c->pops_stale) return TLB_OK;
    k_materialize<L, MODE><<<blocks(c->N, 256), 256, 0, c->stream>>>(
        geo(c), c->ptr<Real>(c->L.M), c->ptr<Store>(c->L.lo[c->cur]), c->ptr<Rest>(c->L.rest[c->cur]));
    TLB_LAUNCHED(c, "k_materialize");
    c->pops_stale = false;
    return TLB_OK;
  }

  // the moments of the streamed populations: pulled from the population
  // buffer, or (moment storage) rebuilt from the stored moments
  static tlb_status launch_moments(Ctx* c, const LBArgs<MODE>& la, cudaStream_t s) {
    if (c->moments() && !c->state_in_pops) {
      // tiles of 32 x 4 columns (2D: 64) walking 16 planes
      constexpr int RX = L::DIM == 3 ? 32 : 64, RY = L::DIM == 3 ? 4 : 1;
      LBArgs<MODE> lr = la;
      lr.zc = 16;
      const dim3 grid(blocks(c->nx, RX), blocks(c->ny, RY), blocks(c->nz, lr.zc));
      k_moments_recon_tiled<L, MODE, RX, RY><<<grid, RX * RY, 0, s>>>(lr);
      TLB_LAUNCHED(c, "k_moments_recon");
    } else {
      // 16-bit storage: 128-thread blocks, finer grains around the membrane
      // kernels that run beside this one (measured 0.262 -> 0.255 ms per
      // step on the 128^3 capsule; FP32 steps were slower with them)
      const int bt = sizeof(Store) == 2 ? 128 : 256;
      k_moments<L, MODE><<<blocks(c->N, bt), bt, 0, s>>>(la);
      TLB_LAUNCHED(c, "k_moments");
    }
    return TLB_OK;
  }

  tlb_status profile_now(Ctx* c) override {
    if (c->nn == 0) return TLB_OK;
    cudaStream_t s = c->stream;
    IBArgs<Real> ia = ibargs(c);
    tlb_status st = snapshot_box(c, ia, s, true);
    if (st == TLB_OK) st = ibm_positions(c, ia, s);
    if (st == TLB_OK) st = ibm_band(c, ia, s);
    c->box_stale = true;  // the next step recomputes the box of these markers
    return st;
  }

  tlb_status init_from_moments(Ctx* c) override {
    cudaStream_t s = c->stream;
    tlb_status pst = profile_now(c);
    if (pst != TLB_OK) return pst;
    Real* uf = c->ptr<Real>(c->L.ftot);  // u = 0
    TLB_CUDA(cudaMemsetAsync(c->ptr<char>(c->L.ftot), 0, c->L.ftot.bytes, s));
    Geo G = geo(c);
    LBArgs<MODE> la = lbargs(c, c->cur);
    Real* mu = c->ptr<Real>(c->L.mu);
    Real *rho = c->ptr<Real>(c->L.rho), *phi = c->ptr<Real>(c->L.phi), *psi = c->ptr<Real>(c->L.psi);
    k_mu_global<L, MODE><<<blocks(c->N, 256), 256, 0, s>>>(G, la.fe, rho, phi, psi, la.I, mu);
    TLB_LAUNCHED(c, "k_mu_global");
    k_init_eq<L, MODE><<<blocks(c->N, 256), 256, 0, s>>>(G, rho, phi, psi, uf, mu, la.gphi, la.gpsi,
                                                          c->ptr<Store>(c->L.lo[c->cur]),
                                                          c->ptr<Rest>(c->L.rest[c->cur]));
    TLB_LAUNCHED(c, "k_init_eq");
    tlb_status rs = residual_launch(c);
    if (rs != TLB_OK) return rs;
    TLB_CUDA(cudaStreamSynchronize(s));
    c->t = 0;
    c->t_snap = 0;
    c->initialised = true;
    c->state_in_pops = true;
    c->pops_stale = false;
    return TLB_OK;
  }

  static ResPtrs resptrs(Ctx* c, unsigned long long* res) {
    return {c->ptr<double>(c->L.snap), c->ptr<double>(c->L.xsnap), res};
  }

  tlb_status residual_launch(Ctx* c) override {
    cudaStream_t s = c->stream;
    if (tlb_status st = sync_pops(c); st != TLB_OK) return st;
    TLB_CUDA(cudaMemsetAsync(c->ptr<char>(c->L.res), 0, c->L.res.bytes, s));
    const unsigned nb = blocks(c->N, 256) + blocks(c->nn, 256);
    k_residual<L, MODE><<<nb, 256, 0, s>>>(geo(c), c->ptr<Store>(c->L.lo[c->cur]), c->ptr<Rest>(c->L.rest[c->cur]),
                                           c->ptr<double>(c->L.X), c->nn,
                                           resptrs(c, c->ptr<unsigned long long>(c->L.res)));
    TLB_LAUNCHED(c, "k_residual");
    return TLB_OK;
  }

  template <int TXv, int TYv, int FORM>
  static tlb_status collide_tile(Ctx* c, LBArgs<MODE>& la, cudaStream_t s) {
    dim3 grid(blocks(c->nx, TXv), blocks(c->ny, TYv), blocks(c->nz, c->tiles_zc));
    k_collide<L, MODE, TXv, TYv, FORM><<<grid, collide_block<FORM, TXv, TYv>(), 0, s>>>(la);
    TLB_LAUNCHED(c, "k_collide");
    return TLB_OK;
  }

  // the collide in the context's variant (tile shape and form)
  static tlb_status collide(Ctx* c, LBArgs<MODE>& la, cudaStream_t s) {
    return collide_variant<L>(c->tile_variant, [&](auto tx, auto ty, auto fm) {
      return collide_tile<decltype(tx)::value, decltype(ty)::value, decltype(fm)::value>(c, la, s);
    });
  }

  // Choose the collide tile shape and z chunk by timing the kernel on the
  // current state (it only reads the current buffer, so repeats are harmless).
  tlb_status autotune(Ctx* c, int* variant, int* zc) override {
    cudaStream_t s = c->stream;
    LBArgs<MODE> la = lbargs(c, c->cur);
    la.jm = c->ptr<Real>(c->L.jm);  // every variant's input, the tau = 1 forms' too
    if (tlb_status st = launch_moments(c, la, s); st != TLB_OK) return st;
    // moment storage: the timed collides store into the idle population
    // buffer, not into the state
    if (c->moments()) la.mst = c->ptr<Real>(c->L.lo[1 - c->cur]);
    cudaEvent_t e0, e1;
    TLB_CUDA(cudaEventCreate(&e0));
    TLB_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bv = c->tile_variant, bz = c->tiles_zc;
    const std::vector<int> zcs = z_chunk_candidates(c->nz);
    for (int v = 0; v < COLLIDE_NVAR; ++v)
      for (const int zcv : zcs) {
        if (!c->variant_ok(v)) continue;
        c->tile_variant = v;
        c->tiles_zc = zcv;
        la.zc = c->tiles_zc;
        tlb_status st = collide(c, la, s);  // warm
        float tmin = 1e30f;
        for (int r = 0; r < 2 && st == TLB_OK; ++r) {
          cudaEventRecord(e0, s);
          st = collide(c, la, s);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          tmin = fminf(tmin, ms);
        }
        if (st != TLB_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
        if (tmin < best) { best = tmin; bv = v; bz = c->tiles_zc; }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tile_variant = bv;
    c->tiles_zc = bz;
    if (variant) *variant = bv;
    if (zc) *zc = bz;
    TLB_CUDA(cudaStreamSynchronize(s));
    return TLB_OK;
  }

  static tlb_status mark(Ctx* c, int k) {
    if (c->prof) TLB_CUDA(cudaEventRecord(c->prof->ev[k], c->stream));
    return TLB_OK;
  }

  static tlb_status collect(Ctx* c) {
    if (!c->prof) return TLB_OK;
    TLB_CUDA(cudaEventSynchronize(c->prof->ev[4]));
    for (int k = 0; k < 4; ++k) {
      float ms = 0;
      TLB_CUDA(cudaEventElapsedTime(&ms, c->prof->ev[k], c->prof->ev[k + 1]));
      c->prof_ms[k] += ms;
    }
    return TLB_OK;
  }

  // n steps; runs of GRAPH_STEPS steps replay a captured graph where the
  // step qualifies (see graph_ready)
  tlb_status step(Ctx* c, long n) override {
    while (n > 0) {
      if (n >= Ctx::GRAPH_STEPS && graph_ready(c)) {
        tlb_status st = replay(c);
        if (st != TLB_OK) return st;
        n -= Ctx::GRAPH_STEPS;
        continue;
      }
      // direct launches until a step qualifies, the rest at the end
      const long k = (n >= Ctx::GRAPH_STEPS && c->graphs && !c->prof) ? 1 : n;
      tlb_status st = step_direct(c, k);
      if (st != TLB_OK) return st;
      n -= k;
    }
    return TLB_OK;
  }

  // A step replays from a graph when it launches the same work every time:
  // no phase profile, no markers set from outside since the last step (their
  // box is rebuilt first) and, with moment storage, the state in the stored
  // moments (the first step after populations were written rebuilds them).
  bool graph_ready(Ctx* c) const {
    return c->graphs && !c->prof && !c->box_stale && !(c->moments() && c->state_in_pops);
  }

  // Launch the graph of the current buffer, capturing it first if missing or
  // captured with another collide variant.  A replay advances the state by
  // GRAPH_STEPS (an even number: the buffer index comes back).
  tlb_status replay(Ctx* c) {
    const int k = c->cur;
    if (!c->gstream) {
      TLB_CUDA(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
      TLB_CUDA(cudaEventCreateWithFlags(&c->ev_gin, cudaEventDisableTiming));
      TLB_CUDA(cudaEventCreateWithFlags(&c->ev_gout, cudaEventDisableTiming));
    }
    cudaStream_t user = c->stream;
    TLB_CUDA(cudaEventRecord(c->ev_gin, user));
    TLB_CUDA(cudaStreamWaitEvent(c->gstream, c->ev_gin, 0));
    if (!c->gexec[k] || c->gsig[k][0] != c->tile_variant || c->gsig[k][1] != c->tiles_zc) {
      if (c->gexec[k]) {  // (after its last replay has finished)
        TLB_CUDA(cudaStreamSynchronize(c->gstream));
        cudaGraphExecDestroy(c->gexec[k]);
        c->gexec[k] = nullptr;
      }
      // capture without executing: the host-side state is put back after
      const int cur0 = c->cur;
      const long t0 = c->t, l0 = c->launches;
      const bool sp0 = c->state_in_pops, ps0 = c->pops_stale;
      TLB_CUDA(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
      c->capturing = true;
      c->stream = c->gstream;
      tlb_status st = step_direct(c, Ctx::GRAPH_STEPS);
      c->stream = user;
      c->capturing = false;
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(c->gstream, &g);
      c->glaunch[k] = c->launches - l0;
      c->cur = cur0;
      c->t = t0;
      c->launches = l0;
      c->state_in_pops = sp0;
      c->pops_stale = ps0;
      if (st == TLB_OK) st = cuda_check(ce, "step graph capture");
      if (st == TLB_OK) st = cuda_check(cudaGraphInstantiate(&c->gexec[k], g, 0), "step graph instantiate");
      if (g) cudaGraphDestroy(g);
      if (st != TLB_OK) {
        c->gexec[k] = nullptr;
        c->graphs = false;  // direct launches from here on
        cudaEventRecord(c->ev_interp, user);
        return st;
      }
      c->gsig[k][0] = c->tile_variant;
      c->gsig[k][1] = c->tiles_zc;
    }
    TLB_CUDA(cudaGraphLaunch(c->gexec[k], c->gstream));
    TLB_CUDA(cudaEventRecord(c->ev_gout, c->gstream));
    TLB_CUDA(cudaStreamWaitEvent(user, c->ev_gout, 0));
    // the events recorded inside the capture stand for graph nodes: the one
    // a direct step waits on before recording it is recorded again here
    TLB_CUDA(cudaEventRecord(c->ev_interp, user));
    c->launches += c->glaunch[k];
    c->t += Ctx::GRAPH_STEPS;
    if (c->moments()) {
      c->state_in_pops = false;
      c->pops_stale = true;
    }
    return TLB_OK;
  }

  tlb_status step_direct(Ctx* c, long n) {
    cudaStream_t s = c->stream;
    const long long N = c->N;
    tlb_status st;
    // Pipelined: the interpolation and advection of a step runs on the side
    // stream beside the next step's moments (which read the populations
    // only); the next step's marker work waits for it there.  The phase
    // profile keeps every kernel on the main stream.
    const bool pipe = c->nn > 0 && !c->prof;
    for (long k = 0; k < n; ++k) {
      LBArgs<MODE> la = lbargs(c, c->cur);
      IBArgs<Real> ia = ibargs(c);
      const bool fresh = c->box_stale;  // markers set from outside since the last step
      c->box_stale = false;
      if ((st = mark(c, 0)) != TLB_OK) return st;
      if (c->nn > 0) {  // fork: position-only membrane work on the two side streams
        // The step's marker box: after markers set from outside it is rebuilt
        // (with the coordinate split the side streams read) before the fork;
        // otherwise it is the previous advection's accumulator, copied on the
        // side stream after that advection.
        const bool box_on_side = pipe && !fresh;
        if (!box_on_side && (st = snapshot_box(c, ia, s, fresh)) != TLB_OK) return st;
        TLB_CUDA(cudaEventRecord(c->ev_fork, s));
        TLB_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        TLB_CUDA(cudaStreamWaitEvent(c->side2, c->ev_fork, 0));
        // the previous advection (a graph's first step follows the whole
        // previous launch on the caller's stream instead)
        if (pipe && !(c->capturing && k == 0)) TLB_CUDA(cudaStreamWaitEvent(c->side2, c->ev_interp, 0));
        if ((st = ibm_positions(c, ia, c->side, box_on_side)) != TLB_OK) return st;
        if ((st = ibm_bins(c, ia, c->side2)) != TLB_OK) return st;
        TLB_CUDA(cudaEventRecord(c->ev_bins, c->side2));
      }
      if ((st = launch_moments(c, la, s)) != TLB_OK) return st;
      if ((st = mark(c, 1)) != TLB_OK) return st;
      // the profile, coupling sums and spreading need psi(t) and the
      // position work: they follow the moments, then the whole lattice is
      // collided in one launch
      if (c->nn > 0) {
        TLB_CUDA(cudaEventRecord(c->ev_join, c->side));
        TLB_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
        TLB_CUDA(cudaStreamWaitEvent(s, c->ev_bins, 0));
        // (in order: running the fill beside the spreading, or splitting the
        // collide to overlap this work, measured slower)
        // (the column fill only after markers were set from outside: between
        // fresh starts the band keeps the cells beyond dc)
        if ((st = launch_band(c, ia, s)) != TLB_OK) return st;
        if (fresh && (st = launch_fill(c, ia, s)) != TLB_OK) return st;
        if ((st = ibm_spread(c, ia, s)) != TLB_OK) return st;
      }
      if ((st = mark(c, 2)) != TLB_OK) return st;
      if ((st = collide(c, la, s)) != TLB_OK) return st;
      if ((st = mark(c, 3)) != TLB_OK) return st;
      if (c->nn > 0) {
        cudaStream_t si = s;
        if (pipe) {
          TLB_CUDA(cudaEventRecord(c->ev_coll, s));
          TLB_CUDA(cudaStreamWaitEvent(c->side, c->ev_coll, 0));
          si = c->side;
        }
        k_interp_advect<L, MODE><<<blocks((long long)c->nn * 32, 128), 128, 0, si>>>(ia, la.lo_dst);
        TLB_LAUNCHED(c, "k_interp_advect");
        if (pipe) TLB_CUDA(cudaEventRecord(c->ev_interp, c->side));
      }
      if ((st = mark(c, 4)) != TLB_OK) return st;
      if ((st = collect(c)) != TLB_OK) return st;
      c->cur = 1 - c->cur;
      c->t += 1;
      if (c->moments()) {  // the state is the stored moments from here on
        c->state_in_pops = false;
        c->pops_stale = true;
      }
    }
    if (pipe && n > 0) TLB_CUDA(cudaStreamWaitEvent(s, c->ev_interp, 0));  // all of it on the caller's stream
    return TLB_OK;
  }

  tlb_status read_field(Ctx* c, int field, double* dst, size_t nvals) override {
    cudaStream_t s = c->stream;
    const long long N = c->N;
    double* rb = c->ptr<double>(c->L.rb);
    const size_t need = field == TLB_FIELD_U ? 3 * (size_t)N : (size_t)N;
    if (nvals < need) { set_error("read_field: buffer too small"); return TLB_ERR_ARG; }
    if (tlb_status st = sync_pops(c); st != TLB_OK) return st;
    // the field is formed on the device, only its values cross to the host
    if (field == TLB_FIELD_I) {
      k_to_double<Real><<<blocks(N, 256), 256, 0, s>>>(c->ptr<Real>(c->L.I), N, rb);
      TLB_LAUNCHED(c, "k_to_double");
    } else {
      k_fields<L, MODE><<<blocks(N, 256), 256, 0, s>>>(geo(c), c->ptr<Store>(c->L.lo[c->cur]),
                                                        c->ptr<Rest>(c->L.rest[c->cur]), field, rb);
      TLB_LAUNCHED(c, "k_fields");
    }
    TLB_CUDA(cudaMemcpyAsync(dst, rb, need * sizeof(double), cudaMemcpyDeviceToHost, s));
    TLB_CUDA(cudaStreamSynchronize(s));
    return TLB_OK;
  }

  // Populations are stored post-collision; the caller's view is the streamed
  // (pre-collision) state.  The conversion runs on the host: it is I/O, not
  // part of the time step.
  static double h2d(double v) { return v; }
  static double h2d(float v) { return v; }
  static double h2d(__half v) { return (double)__half2float(v); }
  static double h2d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
  static void d2h(double v, double& o) { o = v; }
  static void d2h(double v, float& o) { o = (float)v; }
  static void d2h(double v, __half& o) { o = __float2half_rn((float)v); }
  static void d2h(double v, __nv_bfloat16& o) { o = __float2bfloat16_rn((float)v); }

  static long long hwrap(long long a, long long n) { return ((a % n) + n) % n; }

  tlb_status read_pops(Ctx* c, double* dst) override {
    cudaStream_t s = c->stream;
    if (tlb_status st = sync_pops(c); st != TLB_OK) return st;
    const long long N = c->N, P = c->P;
    std::vector<Store> lo((size_t)(3 * L::Q - 2) * P);
    std::vector<Rest> rest((size_t)2 * P);
    TLB_CUDA(cudaMemcpyAsync(lo.data(), c->ptr<Store>(c->L.lo[c->cur]), lo.size() * sizeof(Store), cudaMemcpyDeviceToHost, s));
    TLB_CUDA(cudaMemcpyAsync(rest.data(), c->ptr<Rest>(c->L.rest[c->cur]), rest.size() * sizeof(Rest), cudaMemcpyDeviceToHost, s));
    TLB_CUDA(cudaStreamSynchronize(s));
    for (long long n = 0; n < N; ++n) {
      long long x = n % c->nx, y = (n / c->nx) % c->ny, z = n / ((long long)c->nx * c->ny);
      for (int i = 0; i < L::Q; ++i) {
        long long sz = z - L::cz(i), src;
        int ii = i;
        if (c->p.wall_last && (sz < 0 || sz >= c->nz)) { src = n; ii = L::opp(i); }
        else src = (hwrap(sz, c->nz) * c->ny + hwrap(y - L::cy(i), c->ny)) * c->nx + hwrap(x - L::cx(i), c->nx);
        dst[(long long)i * N + n] = h2d(lo[(size_t)plane_f<L>(ii) * P + src]) + L::w(ii);
        dst[(long long)(L::Q + i) * N + n] = ii == 0 ? h2d(rest[src]) : h2d(lo[(size_t)plane_g<L>(ii) * P + src]);
        dst[(long long)(2 * L::Q + i) * N + n] = ii == 0 ? h2d(rest[P + src]) : h2d(lo[(size_t)plane_h<L>(ii) * P + src]);
      }
    }
    return TLB_OK;
  }

  tlb_status write_pops(Ctx* c, const double* src_in) override {
    cudaStream_t s = c->stream;
    const long long N = c->N, P = c->P;
    std::vector<Store> lo((size_t)(3 * L::Q - 2) * P);
    std::vector<Rest> rest((size_t)2 * P);
    for (long long n = 0; n < N; ++n) {
      long long x = n % c->nx, y = (n / c->nx) % c->ny, z = n / ((long long)c->nx * c->ny);
      for (int i = 0; i < L::Q; ++i) {
        long long tz = z + L::cz(i), src;
        int ii = i;
        if (c->p.wall_last && (tz < 0 || tz >= c->nz)) { src = n; ii = L::opp(i); }
        else src = (hwrap(tz, c->nz) * c->ny + hwrap(y + L::cy(i), c->ny)) * c->nx + hwrap(x + L::cx(i), c->nx);
        d2h(src_in[(long long)ii * N + src] - L::w(ii), lo[(size_t)plane_f<L>(i) * P + n]);
        if (ii == 0) {
          d2h(src_in[(long long)L::Q * N + src], rest[n]);
          d2h(src_in[(long long)2 * L::Q * N + src], rest[P + n]);
        } else {
          d2h(src_in[(long long)(L::Q + ii) * N + src], lo[(size_t)plane_g<L>(i) * P + n]);
          d2h(src_in[(long long)(2 * L::Q + ii) * N + src], lo[(size_t)plane_h<L>(i) * P + n]);
        }
      }
    }
    TLB_CUDA(cudaMemcpyAsync(c->ptr<Store>(c->L.lo[c->cur]), lo.data(), lo.size() * sizeof(Store), cudaMemcpyHostToDevice, s));
    TLB_CUDA(cudaMemcpyAsync(c->ptr<Rest>(c->L.rest[c->cur]), rest.data(), rest.size() * sizeof(Rest), cudaMemcpyHostToDevice, s));
    TLB_CUDA(cudaStreamSynchronize(s));
    c->initialised = true;
    c->state_in_pops = true;  // (moment storage: the next step pulls them)
    c->pops_stale = false;
    return TLB_OK;
  }

  // Contact angles (tlb_measure.cuh).  Scratch: phi in the read-back
  // buffer; marker values, edge angles and the per-capsule results in the
  // population buffer that the next step writes (idle between steps).
  tlb_status contact_angle(Ctx* c, double* out) override {
    cudaStream_t s = c->stream;
    const long long N = c->N;
    const int nedge = c->NV == 2 ? c->nn : c->nedge;
    const size_t need = (size_t)(4 * c->nn + nedge + 4 * c->ncap) * sizeof(double) + (size_t)nedge * sizeof(int);
    if (c->ncap == 0) return TLB_OK;
    if (need > c->L.lo[1 - c->cur].bytes) { set_error("contact_angle: scratch too small"); return TLB_ERR_ARG; }
    if (tlb_status st = sync_pops(c); st != TLB_OK) return st;
    double* phi = c->ptr<double>(c->L.rb);
    k_fields<L, MODE><<<blocks(N, 256), 256, 0, s>>>(geo(c), c->ptr<Store>(c->L.lo[c->cur]),
                                                      c->ptr<Rest>(c->L.rest[c->cur]), TLB_FIELD_PHI, phi);
    TLB_LAUNCHED(c, "k_fields");
    double* sc = c->ptr<double>(c->L.lo[1 - c->cur]);
    AngleArgs a;
    a.G = geo(c);
    a.dim = c->p.dim;
    a.nn = c->nn;
    a.NV = c->NV;
    a.X = c->ptr<double>(c->L.X);
    a.phi = phi;
    a.E = c->ptr<int>(c->L.E);
    a.inc_off = c->ptr<int>(c->L.inc_off);
    a.inc = c->ptr<int>(c->L.inc);
    a.rnext = c->ptr<int>(c->L.rnext);
    a.rprev = c->ptr<int>(c->L.rprev);
    a.edges = c->ptr<int>(c->L.edges);
    a.ncap = c->ptr<int>(c->L.ncap);
    a.nedge = nedge;
    a.mk = sc;
    a.ang = sc + 4 * c->nn;
    double* res = a.ang + nedge;
    a.ecapo = reinterpret_cast<int*>(res + 4 * c->ncap);
    k_marker_phi<<<blocks(c->nn, 128), 128, 0, s>>>(a);
    TLB_LAUNCHED(c, "k_marker_phi");
    k_contact_edges<L><<<blocks(nedge, 128), 128, 0, s>>>(a);
    TLB_LAUNCHED(c, "k_contact_edges");
    k_contact_reduce<<<c->ncap, 256, 0, s>>>(a.ang, a.ecapo, nedge, res);
    TLB_LAUNCHED(c, "k_contact_reduce");
    TLB_CUDA(cudaMemcpyAsync(out, res, 4 * c->ncap * sizeof(double), cudaMemcpyDeviceToHost, s));
    TLB_CUDA(cudaStreamSynchronize(s));
    return TLB_OK;
  }

  tlb_status diagnostics(Ctx* c, tlb_diag* out) override {
    if (tlb_status st = sync_pops(c); st != TLB_OK) return st;
    return fp64_diagnostics<L, MODE>(c, c->ptr<double>(c->L.part), 1024, c->ptr<double>(c->L.meas), out);
  }
};
