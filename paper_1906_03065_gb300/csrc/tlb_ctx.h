// Host-side context of the library: the arena layout and the per-context
// state.  The caller's arena is carved into fixed regions once, at
// tlb_create; no other device memory is ever allocated.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tlb.h"

// Collide variants: 3 tile shapes x 4 register forms, v = 3 form + tile,
// the smallest tile in a fifth form (v = 12), and the 3 tiles in the two
// forms of the tau = 1 collide (v = 13..18, see variant_t1).
constexpr int COLLIDE_NVAR = 32;
constexpr bool variant_t1(int v) { return (v >= 13 && v <= 18) || v >= 22; }
// variants 22..27 and 30, 31: the tau = 1 collide with two x-adjacent cells
// per thread; 28..31 are the tau = 1 forms on 32 x 16 tiles
constexpr bool variant_pair(int v) { return (v >= 22 && v <= 27) || v == 30 || v == 31; }
// variants 19..21: the general collide with the pressure-tensor force
constexpr bool variant_pt(int v) { return v >= 19 && v <= 21; }

// z-chunk lengths the collide autotuner tries: every distinct ceil(nz / m)
// of at least 4 planes (each gives another grid, so another fill of the
// last wave of blocks).
inline std::vector<int> z_chunk_candidates(int nz) {
  std::vector<int> v;
  for (int m = 1;; ++m) {
    const int zc = (nz + m - 1) / m;
    if (v.empty() || v.back() != zc) v.push_back(zc);
    if (zc <= 4) break;
  }
  return v;
}

struct Ctx;

struct ImplBase {
  virtual ~ImplBase() {}
  virtual tlb_status init_fields(Ctx* c, const double* C, const double* u) = 0;
  virtual tlb_status step(Ctx* c, long n) = 0;
  virtual tlb_status read_field(Ctx* c, int field, double* dst, size_t n) = 0;
  virtual tlb_status read_pops(Ctx* c, double* dst) = 0;
  virtual tlb_status write_pops(Ctx* c, const double* src) = 0;
  virtual tlb_status diagnostics(Ctx* c, tlb_diag* out) = 0;
  virtual tlb_status autotune(Ctx* c, int* variant, int* zc) = 0;
  // launches the residual kernel into c->L.res (zeroed first); no sync
  virtual tlb_status residual_launch(Ctx* c) = 0;
  // initial state from the rho, phi, psi moment arrays as they stand and the
  // current marker positions (profile, u = 0, equilibrium populations)
  virtual tlb_status init_from_moments(Ctx* c) = 0;
  // profile I (with owners and distances) of the current marker positions
  virtual tlb_status profile_now(Ctx* c) = 0;
  // contact angle of every capsule with phi = 0: out[cap] = {mean, min,
  // max, contact points}; synchronises
  virtual tlb_status contact_angle(Ctx* c, double* out) = 0;
  // moment storage: write the populations the stored moments stand for into
  // the current population buffer if it is stale (no-op otherwise)
  virtual tlb_status sync_pops(Ctx* c) = 0;
};

// CUDA events bracketing the phases of a step when profiling.
struct PhaseEvents {
  cudaEvent_t ev[5];
  bool on = false;
};

// Sizes in bytes of the precision-dependent element types.
struct TypeSizes {
  size_t real, store, rest;
};

// One region of the arena.
struct Region {
  size_t off = 0, bytes = 0;
};

struct Layout {
  // lattice
  Region lo[2], rest[2];
  Region rho, phi, psi, jm, M, I, dsel, own, key, fib, ftot, mu, rb;
  // membranes
  Region X, E, ecap, ncap, cap_par, ds0, rprev, rnext, A0, G0i, inc_off, inc, adj, edges, ring_off, ring;
  Region en, vn, erel, eorg, ecst, xo, xr, skc, capr, ncpl, F, box;
  Region bcnt, bprev, bcur, boff, blist, bact, ctr, bflag;
  // misc
  Region status, part, meas;
  // equilibrium residual: reference phi, psi and marker positions, maxima
  Region snap, xsnap, res;
  size_t total = 0;
};

struct HostMem {
  int kind, nn, ne;
  std::vector<double> X0;  // internal coordinates, unwrapped along edges
  std::vector<int> E;
  double ks, kb, G, C;
};

struct Ctx {
  tlb_params p;
  // the tau = 1 collide applies: tau = tau_phi = tau_psi = 1 and the exact
  // difference method (every post-collision population is an equilibrium)
  bool t1_ok() const {
    return p.tau == 1.0 && p.tau_phi == 1.0 && p.tau_psi == 1.0 && p.forcing == TLB_FORCE_EDM &&
           p.force_form == TLB_FE_POTENTIAL;
  }
  // a collide variant this context can run: the pressure-tensor variants for
  // the pressure-tensor force only, the tau = 1 ones only where they apply,
  // and with moment storage only the tau = 1 ones
  bool variant_ok(int v) const {
    if (variant_pt(v) != (p.force_form == TLB_FE_PRESSURE_TENSOR)) return false;
    if (variant_pair(v) && nx % 2 != 0) return false;  // pairs never straddle a row
    if (variant_t1(v)) return t1_ok();
    return !moments();
  }
  // moment storage (TLB_STATE_MOMENTS): the state is the moment buffer M,
  // except after an initialisation or a write of populations, which the
  // next step pulls as populations (state_in_pops); the population buffer
  // is refreshed from M for readers when it is stale
  bool moments() const { return p.state == TLB_STATE_MOMENTS; }
  bool state_in_pops = true;
  bool pops_stale = false;
  int Q = 0;
  int nx = 0, ny = 0, nz = 0;  // internal sizes (2D: nx, 1, ny)
  long long N = 0, P = 0;
  TypeSizes ts{};
  Layout L;
  char* base = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;   // membrane work that overlaps the moments: geometry
                                 // and the distance scatter
  cudaStream_t side2 = nullptr;  // elastic forces and brick binning, beside `side`
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_bins = nullptr, ev_coll = nullptr, ev_interp = nullptr;
  int nsm = 1;  // streaming multiprocessors of the device
  int cur = 0;  // population buffer holding the current state
  long t = 0;
  long t_snap = 0;  // step of the residual's reference state
  bool initialised = false;
  bool box_stale = false;  // markers were overwritten: recompute the marker box
  long launches = 0;
  // membranes
  std::vector<HostMem> mems;
  int nn = 0, ne = 0, NV = 0, ncap = 0, nedge = 0;
  int nbx = 0, nby = 0, nbz = 0, nbricks = 0;
  int tiles_zc = 16;
  int tile_variant = 0;  // collide tile shape and form (see collide_variant)
  PhaseEvents* prof = nullptr;  // non-null while tlb_profile_steps runs
  double prof_ms[4] = {0, 0, 0, 0};
  ImplBase* impl = nullptr;
  // Step graphs: GRAPH_STEPS steps captured from the context's streams and
  // replayed as one graph launch, one graph per starting population buffer;
  // a graph holds the collide variant and z chunk it was captured with.
  static constexpr int GRAPH_STEPS = 8;
  bool graphs = false;         // replay captured steps where a step qualifies
  bool capturing = false;      // the steps being issued are captured
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // graphs are captured on and replayed from a stream of the context's own
  // (the caller's stream may be the legacy default stream, which cannot be
  // captured), ordered after and before the caller's stream by two events
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_gin = nullptr, ev_gout = nullptr;
  int gsig[2][2] = {{-1, -1}, {-1, -1}};  // (tile_variant, tiles_zc) of each graph
  long glaunch[2] = {0, 0};    // kernel launches one replay makes
  void drop_graphs() {
    for (int k = 0; k < 2; ++k) {
      if (gexec[k]) cudaGraphExecDestroy(gexec[k]);
      gexec[k] = nullptr;
      gsig[k][0] = gsig[k][1] = -1;
    }
  }

  template <class T> T* ptr(const Region& r) const { return reinterpret_cast<T*>(base + r.off); }

  ~Ctx() {
    if (gstream) cudaStreamSynchronize(gstream);
    drop_graphs();
    if (ev_gin) cudaEventDestroy(ev_gin);
    if (ev_gout) cudaEventDestroy(ev_gout);
    if (gstream) cudaStreamDestroy(gstream);
    if (side) cudaStreamSynchronize(side);
    if (side2) cudaStreamSynchronize(side2);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_bins) cudaEventDestroy(ev_bins);
    if (ev_coll) cudaEventDestroy(ev_coll);
    if (ev_interp) cudaEventDestroy(ev_interp);
    if (side) cudaStreamDestroy(side);
    if (side2) cudaStreamDestroy(side2);
  }
};

struct Batch;

struct BatchBase {
  virtual ~BatchBase() {}
  virtual tlb_status step(Batch* b, long n) = 0;
  // launches the residual of every active instance into its slot of b->res
  // (zeroed first); no sync
  virtual tlb_status residual(Batch* b) = 0;
  virtual tlb_status autotune(Batch* b, int* variant, int* zc) = 0;
  // n steps with direct launches, device time of each of the six phases
  // summed into ms[0..5]; synchronises
  virtual tlb_status profile(Batch* b, long n, double* ms) = 0;
};

// A batch of independent contexts of one lattice type and storage, stepped
// together (see tlb_batch.cuh).  The instances live in sub-arenas of the
// batch arena, followed by the batch's own tables.
struct Batch {
  static constexpr int NPH = 7;      // six phases of a step + the residual
  static constexpr int MAXOPS = 4;   // kernel bodies per phase
  static constexpr size_t ARGS_BYTES = 1024;  // bound on one instance's argument record
  std::vector<Ctx*> inst;
  std::vector<int> act;  // active instances, ascending
  int dim = 0, storage = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // capture stream of the step graph
  char* base = nullptr;
  size_t bytes = 0;
  Region targs[2], vg, res;
  std::vector<int> band_blocks, spread_blocks;  // virtual grids of the box-sized ops
  int ph_ent[NPH] = {0}, ph_total[NPH] = {0}, ph_grid[NPH] = {0};
  cudaGraphExec_t graph = nullptr;
  bool graph_dirty = true;
  long graph_launches = 0;  // kernels in one launch of the step graph
  int tile_variant = 0, zc = 16;
  long launches = 0;
  BatchBase* impl = nullptr;

  template <class T> T* ptr(const Region& r) const { return reinterpret_cast<T*>(base + r.off); }

  ~Batch() {
    if (stream) cudaStreamSynchronize(stream);
    if (graph) cudaGraphExecDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    for (Ctx* c : inst) delete c;
  }
};

void set_error(const std::string& msg);
tlb_status cuda_check(cudaError_t e, const char* what);
#define TLB_CUDA(call)                                              \
  do {                                                              \
    tlb_status _s = cuda_check((call), #call);                      \
    if (_s != TLB_OK) return _s;                                    \
  } while (0)
#define TLB_LAUNCHED(ctx, what)                                     \
  do {                                                              \
    (ctx)->launches++;                                              \
    tlb_status _s = cuda_check(cudaGetLastError(), what);           \
    if (_s != TLB_OK) return _s;                                    \
  } while (0)

ImplBase* make_impl_d2q9_f64();
ImplBase* make_impl_d2q9_f32();
ImplBase* make_impl_d3q19_f32();
ImplBase* make_impl_d3q19_f16();
ImplBase* make_impl_d3q19_bf16();
BatchBase* make_batch_impl_d2q9_f64();
BatchBase* make_batch_impl_d2q9_f32();
BatchBase* make_batch_impl_d3q19_f32();
BatchBase* make_batch_impl_d3q19_f16();
BatchBase* make_batch_impl_d3q19_bf16();
