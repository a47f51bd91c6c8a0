// C ABI of libtlb (see include/tlb.h): argument checking, arena layout,
// membrane preprocessing and dispatch to the templated drivers.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "tlb_ctx.h"

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

tlb_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TLB_OK;
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // reported here: not left for the caller's next CUDA call
  return TLB_ERR_CUDA;
}

// ------------------------------------------------------------ small kernels
__global__ void k_reduce_partials(const double* part, int nb, int nq, double* out) {
  __shared__ double sm[256];
  for (int q = 0; q < nq; ++q) {
    double acc = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[q * nb + i];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sm[0];
    __syncthreads();
  }
}

__global__ void k_capsule_measures(const double* X, const int* E, const int* ecap, int ne, int NV, int ncap,
                                   double* out) {
  __shared__ double sa[256], sv[256];
  const int cap = blockIdx.x;
  double A = 0, V = 0;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    if (ecap[e] != cap) continue;
    if (NV == 2) {
      const double* p = X + 3 * E[2 * e];
      const double* q = X + 3 * E[2 * e + 1];
      A += 0.5 * (p[0] * q[2] - q[0] * p[2]);  // internal (x, z) = paper (x, y)
    } else {
      const double* a = X + 3 * E[3 * e];
      const double* b = X + 3 * E[3 * e + 1];
      const double* c = X + 3 * E[3 * e + 2];
      double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
      A += 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
      V += (a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]) / 6.0;
    }
  }
  sa[threadIdx.x] = A;
  sv[threadIdx.x] = V;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sv[threadIdx.x] += sv[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * cap] = sa[0];
    out[2 * cap + 1] = sv[0];
  }
}

__global__ void k_fill_real(float* p, long long n, float v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
__global__ void k_fill_real(double* p, long long n, double v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// ------------------------------------------------------------ validation
static size_t real_size(int storage) { return storage == TLB_F64 ? 8 : 4; }
static size_t store_size(int storage) {
  return storage == TLB_F64 ? 8 : (storage == TLB_F32 ? 4 : 2);
}
static size_t rest_size(int storage) { return storage == TLB_F64 ? 8 : 4; }

static tlb_status check_params(const tlb_params* p, const tlb_membrane_desc* mems, int n_mem) {
  if (!p) { set_error("params is NULL"); return TLB_ERR_ARG; }
  if (p->dim != 2 && p->dim != 3) { set_error("dim must be 2 or 3"); return TLB_ERR_ARG; }
  if (p->storage < TLB_F64 || p->storage > TLB_BF16) { set_error("unknown storage"); return TLB_ERR_ARG; }
  if (p->dim == 2 && p->storage != TLB_F64 && p->storage != TLB_F32) {
    set_error("2D lattices support TLB_F64 and TLB_F32 storage");
    return TLB_ERR_ARG;
  }
  if (p->dim == 3 && p->storage == TLB_F64) { set_error("3D lattices support F32/F16/BF16 storage"); return TLB_ERR_ARG; }
  int nz = p->dim == 3 ? p->nz : 1;
  if (p->nx < 4 || p->ny < 4 || (p->dim == 3 && nz < 4)) { set_error("lattice sides must be >= 4"); return TLB_ERR_ARG; }
  {
    // population offsets (3Q planes of the padded cell count) are 32-bit
    const long long cells = (long long)p->nx * p->ny * nz;
    const long long planes = p->dim == 3 ? 3 * 19 : 3 * 9;
    if ((cells + 64) * planes >= (1ll << 31)) {
      set_error("lattice too large: 3Q x cells must stay below 2^31");
      return TLB_ERR_ARG;
    }
  }
  if (!(p->tau > 0.5 && p->tau_phi > 0.5 && p->tau_psi > 0.5)) { set_error("relaxation times must exceed 1/2"); return TLB_ERR_ARG; }
  if (!(p->alpha > 0) || !(p->dc > 0) || p->dc > 60) { set_error("alpha > 0 and 0 < dc <= 60 required"); return TLB_ERR_ARG; }
  if (p->forcing != TLB_FORCE_EDM && p->forcing != TLB_FORCE_GUO) { set_error("unknown forcing"); return TLB_ERR_ARG; }
  if (p->state != TLB_STATE_POPULATIONS && p->state != TLB_STATE_MOMENTS) { set_error("unknown state"); return TLB_ERR_ARG; }
  if (p->force_form != TLB_FE_POTENTIAL && p->force_form != TLB_FE_PRESSURE_TENSOR) {
    set_error("unknown force_form");
    return TLB_ERR_ARG;
  }
  if (p->state == TLB_STATE_MOMENTS && p->force_form != TLB_FE_POTENTIAL) {
    set_error("TLB_STATE_MOMENTS needs the potential force form");
    return TLB_ERR_ARG;
  }
  if (p->state == TLB_STATE_MOMENTS) {
    if (!(p->tau == 1.0 && p->tau_phi == 1.0 && p->tau_psi == 1.0 && p->forcing == TLB_FORCE_EDM)) {
      set_error("TLB_STATE_MOMENTS needs tau = tau_phi = tau_psi = 1 and TLB_FORCE_EDM");
      return TLB_ERR_ARG;
    }
    if (!(p->storage == TLB_F32 || (p->dim == 2 && p->storage == TLB_F64))) {
      set_error("TLB_STATE_MOMENTS needs FP32 storage (or FP64 in 2D)");
      return TLB_ERR_ARG;
    }
  }
  if (n_mem < 0 || n_mem > 8) { set_error("at most 8 membranes"); return TLB_ERR_ARG; }
  for (int m = 0; m < n_mem; ++m) {
    const tlb_membrane_desc& d = mems[m];
    if ((p->dim == 2) != (d.kind == TLB_MEM_RING2D)) { set_error("membrane kind does not match dim"); return TLB_ERR_ARG; }
    if (d.n_nodes < 3 || !d.X0) { set_error("membrane needs >= 3 nodes and X0"); return TLB_ERR_ARG; }
    if (d.kind == TLB_MEM_TRI3D && (d.n_elems < 4 || !d.elems)) { set_error("triangle membrane needs elems"); return TLB_ERR_ARG; }
    if (d.kind == TLB_MEM_TRI3D && (long long)d.n_elems * n_mem >= (1 << 24)) { set_error("too many elements"); return TLB_ERR_ARG; }
  }
  if (n_mem > 0) {
    // sweep regions of an element must not wrap onto themselves
    int need = 2 * (int)ceil(p->dc) + 8;
    if (p->nx < need || (p->dim == 3 && p->ny < need) || (!p->wall_last && (p->dim == 3 ? nz : p->ny) < need)) {
      set_error("periodic sides must be at least 2*dc + 8 cells when membranes are present");
      return TLB_ERR_ARG;
    }
  }
  return TLB_OK;
}

// ------------------------------------------------------------ membranes
static void preprocess(const tlb_params* p, const tlb_membrane_desc* mems, int n_mem, std::vector<HostMem>& out) {
  out.clear();
  const int n[3] = {p->nx, p->dim == 3 ? p->ny : 1, p->dim == 3 ? p->nz : p->ny};
  const bool wall_z = p->wall_last != 0;
  for (int m = 0; m < n_mem; ++m) {
    const tlb_membrane_desc& d = mems[m];
    HostMem h;
    h.kind = d.kind;
    h.nn = d.n_nodes;
    h.ks = d.ks;
    h.kb = d.kb;
    h.G = d.skalak_G;
    h.C = d.skalak_C;
    std::vector<double> X(3 * h.nn);
    for (int l = 0; l < h.nn; ++l) {
      if (d.kind == TLB_MEM_RING2D) {
        X[3 * l] = d.X0[3 * l];
        X[3 * l + 1] = 0.0;
        X[3 * l + 2] = d.X0[3 * l + 1];
      } else {
        for (int k = 0; k < 3; ++k) X[3 * l + k] = d.X0[3 * l + k];
      }
    }
    int NV = d.kind == TLB_MEM_RING2D ? 2 : 3;
    if (d.kind == TLB_MEM_RING2D) {
      h.ne = h.nn;
      h.E.resize(2 * h.nn);
      for (int l = 0; l < h.nn; ++l) { h.E[2 * l] = l; h.E[2 * l + 1] = (l + 1) % h.nn; }
    } else {
      h.ne = d.n_elems;
      h.E.assign(d.elems, d.elems + 3 * d.n_elems);
    }
    // make the copy contiguous: unwrap every marker along the mesh edges
    std::vector<std::vector<int>> nb(h.nn);
    for (int e = 0; e < h.ne; ++e)
      for (int q = 0; q < NV; ++q) {
        int a = h.E[NV * e + q], b = h.E[NV * e + (q + 1) % NV];
        nb[a].push_back(b);
        nb[b].push_back(a);
      }
    std::vector<char> seen(h.nn, 0);
    h.X0.assign(3 * h.nn, 0.0);
    for (int r = 0; r < h.nn; ++r) {
      if (seen[r]) continue;
      seen[r] = 1;
      for (int k = 0; k < 3; ++k) h.X0[3 * r + k] = X[3 * r + k];
      std::vector<int> st{r};
      while (!st.empty()) {
        int a = st.back();
        st.pop_back();
        for (int b : nb[a]) {
          if (seen[b]) continue;
          seen[b] = 1;
          for (int k = 0; k < 3; ++k) {
            double dlt = X[3 * b + k] - X[3 * a + k];
            if (!(k == 2 && wall_z)) dlt -= n[k] * floor(dlt / n[k] + 0.5);
            h.X0[3 * b + k] = h.X0[3 * a + k] + dlt;
          }
          st.push_back(b);
        }
      }
    }
    out.push_back(h);
  }
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static void plan(const tlb_params* p, const std::vector<HostMem>& mems, Ctx& c) {
  c.p = *p;
  c.Q = p->dim == 3 ? 19 : 9;
  c.nx = p->nx;
  c.ny = p->dim == 3 ? p->ny : 1;
  c.nz = p->dim == 3 ? p->nz : p->ny;
  c.N = (long long)c.nx * c.ny * c.nz;
  c.P = (c.N + 63) / 64 * 64;
  c.ts = {real_size(p->storage), store_size(p->storage), rest_size(p->storage)};
  c.NV = p->dim == 3 ? 3 : 2;
  c.nn = c.ne = c.nedge = 0;
  c.ncap = (int)mems.size();
  for (const HostMem& m : mems) {
    c.nn += m.nn;
    c.ne += m.ne;
    if (m.kind == TLB_MEM_TRI3D) c.nedge += 3 * m.ne / 2;  // closed surface: each edge in two faces
  }
  c.nbx = (c.nx + 3) / 4;
  c.nby = p->dim == 3 ? (c.ny + 3) / 4 : 1;
  c.nbz = (c.nz + 3) / 4;
  c.nbricks = c.nbx * c.nby * c.nbz;
  Layout& L = c.L;
  size_t off = 0;
  auto take = [&](Region& r, size_t bytes) {
    r.off = off;
    r.bytes = bytes;
    off = align256(off + std::max<size_t>(bytes, 1));
  };
  const size_t P = (size_t)c.P, R = c.ts.real;
  for (int b = 0; b < 2; ++b) {
    take(L.lo[b], (size_t)(3 * c.Q - 2) * P * c.ts.store);
    take(L.rest[b], 2 * P * c.ts.rest);
  }
  take(L.rho, P * R);
  take(L.phi, P * R);
  take(L.psi, P * R);
  take(L.jm, 3 * P * R);
  take(L.M, p->state == TLB_STATE_MOMENTS ? 11 * P * R : 0);
  take(L.I, P * R);
  take(L.dsel, P * R);
  take(L.own, P * 4);
  take(L.key, P * 8);
  take(L.fib, 3 * P * R);
  take(L.ftot, 3 * P * R);
  take(L.mu, 3 * P * R);
  take(L.rb, 6 * P * 8);
  const size_t nn = c.nn, ne = c.ne, NV = c.NV;
  take(L.X, 3 * nn * 8);
  take(L.E, NV * ne * 4);
  take(L.ecap, ne * 4);
  take(L.ncap, nn * 4);
  take(L.cap_par, 4 * std::max(1, c.ncap) * 8);
  take(L.ds0, ne * 8);
  take(L.rprev, nn * 4);
  take(L.rnext, nn * 4);
  take(L.A0, ne * 8);
  take(L.G0i, 3 * ne * 8);
  take(L.inc_off, (nn + 1) * 4);
  take(L.inc, NV * ne * 4);
  take(L.adj, 3 * ne * 4);
  take(L.edges, 4 * (size_t)c.nedge * 4);
  take(L.ring_off, (nn + 1) * 4);
  take(L.ring, NV * ne * 4);
  take(L.en, 3 * ne * R);
  take(L.vn, 3 * nn * R);
  take(L.erel, 3 * NV * ne * R);
  take(L.eorg, 3 * ne * 4);
  take(L.ecst, 16 * ne * R);
  take(L.xo, 3 * nn * 4);
  take(L.xr, 3 * nn * R);
  take(L.skc, 5 * ne * R);
  take(L.capr, 4 * std::max(1, c.ncap) * R);
  take(L.ncpl, 3 * nn * 8);
  take(L.F, 3 * nn * R);
  take(L.box, 12 * 4);
  const size_t nb = c.nbricks;
  take(L.bcnt, nb * 4);
  take(L.bprev, nb * 4);
  take(L.bcur, nb * 4);
  take(L.boff, nb * 4);
  take(L.blist, 27 * nn * 4);
  take(L.bact, nb * 4);
  take(L.ctr, 4 * 4);
  take(L.bflag, nb);
  take(L.status, 64);
  take(L.part, 3 * 1024 * 8);
  take(L.meas, 32 * 8);
  take(L.snap, 2 * P * 8);
  take(L.xsnap, 3 * nn * 8);
  take(L.res, 4 * 8);
  L.total = off;
}

// ------------------------------------------------------------ C ABI
extern "C" {

const char* tlb_last_error(void) { return g_err.c_str(); }

tlb_status tlb_state_bytes(const tlb_params* params, const tlb_membrane_desc* mems, int n_mem, size_t* bytes) {
  tlb_status s = check_params(params, mems, n_mem);
  if (s != TLB_OK) return s;
  if (!bytes) { set_error("bytes is NULL"); return TLB_ERR_ARG; }
  std::vector<HostMem> hm;
  preprocess(params, mems, n_mem, hm);
  Ctx c;
  plan(params, hm, c);
  *bytes = c.L.total;
  return TLB_OK;
}

tlb_status tlb_create(const tlb_params* params, const tlb_membrane_desc* mems, int n_mem, void* arena,
                      size_t bytes, void* cuda_stream, void** ctx_out) {
  tlb_status s = check_params(params, mems, n_mem);
  if (s != TLB_OK) return s;
  if (!arena || !ctx_out) { set_error("arena and ctx_out must be non-NULL"); return TLB_ERR_ARG; }
  if (((uintptr_t)arena) & 255) { set_error("arena must be 256-byte aligned"); return TLB_ERR_ARG; }
  Ctx* c = new Ctx();
  preprocess(params, mems, n_mem, c->mems);
  plan(params, c->mems, *c);
  if (bytes < c->L.total) {
    set_error("arena too small: need " + std::to_string(c->L.total) + " bytes");
    delete c;
    return TLB_ERR_ALLOC;
  }
  c->base = (char*)arena;
  c->bytes = bytes;
  c->stream = (cudaStream_t)cuda_stream;
  // z chunk of the plane sweep: long enough to amortise the 4-plane halo,
  // short enough to give a few waves on the 152 SMs
  c->tiles_zc = c->nz >= 64 ? 32 : (c->nz >= 16 ? 8 : c->nz);
  // the tau = 1 collide (no population pull) wherever it applies
  c->tile_variant = params->force_form == TLB_FE_PRESSURE_TENSOR ? 19 : (c->t1_ok() ? 13 : 0);
  switch (params->dim * 10 + params->storage) {
    case 20: c->impl = make_impl_d2q9_f64(); break;
    case 21: c->impl = make_impl_d2q9_f32(); break;
    case 31: c->impl = make_impl_d3q19_f32(); break;
    case 32: c->impl = make_impl_d3q19_f16(); break;
    case 33: c->impl = make_impl_d3q19_bf16(); break;
    default: set_error("unsupported dim/storage"); delete c; return TLB_ERR_ARG;
  }
  cudaStream_t st = c->stream;
  {
    // the membrane work is short and latency bound: give its streams the
    // highest priority so its blocks go first beside the moments kernel
    int lo_prio = 0, hi_prio = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (c->nsm <= 0) c->nsm = 1;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    tlb_status r0 = cuda_check(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi_prio), "side stream");
    if (r0 == TLB_OK)
      r0 = cuda_check(cudaStreamCreateWithPriority(&c->side2, cudaStreamNonBlocking, hi_prio), "side stream");
    if (r0 == TLB_OK) r0 = cuda_check(cudaEventCreateWithFlags(&c->ev_bins, cudaEventDisableTiming), "event");
    if (r0 == TLB_OK) r0 = cuda_check(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "event");
    if (r0 == TLB_OK) r0 = cuda_check(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "event");
    if (r0 == TLB_OK) r0 = cuda_check(cudaEventCreateWithFlags(&c->ev_coll, cudaEventDisableTiming), "event");
    if (r0 == TLB_OK) r0 = cuda_check(cudaEventCreateWithFlags(&c->ev_interp, cudaEventDisableTiming), "event");
    if (r0 != TLB_OK) { delete c; return r0; }
  }
  // zero everything, then set the non-zero initial values
  tlb_status r = cuda_check(cudaMemsetAsync(c->base, 0, c->L.total, st), "memset arena");
  if (r != TLB_OK) { delete c; return r; }
  cudaMemsetAsync(c->ptr<char>(c->L.key), 0xFF, c->L.key.bytes, st);
  cudaMemsetAsync(c->ptr<char>(c->L.own), 0xFF, c->L.own.bytes, st);
  const double Iout = 0.5 * (1.0 + tanh(-params->dc / (2.0 * params->alpha)));
  const long long P = c->P;
  unsigned nb = (unsigned)((P + 255) / 256);
  if (c->ts.real == 8) {
    k_fill_real<<<nb, 256, 0, st>>>(c->ptr<double>(c->L.I), P, Iout);
    k_fill_real<<<nb, 256, 0, st>>>(c->ptr<double>(c->L.dsel), P, -params->dc);
  } else {
    k_fill_real<<<nb, 256, 0, st>>>(c->ptr<float>(c->L.I), P, (float)Iout);
    k_fill_real<<<nb, 256, 0, st>>>(c->ptr<float>(c->L.dsel), P, (float)-params->dc);
  }
  // membranes
  if (c->ncap > 0) {
    std::vector<double> X, cap_par(4 * c->ncap), ds0, A0, G0i;
    std::vector<int> E, ecap, ncap, rprev, rnext, adj, edges;
    std::vector<std::vector<int>> inc(c->nn);
    int noff = 0, eoff = 0;
    for (int m = 0; m < c->ncap; ++m) {
      const HostMem& h = c->mems[m];
      cap_par[m] = h.ks;
      cap_par[c->ncap + m] = h.kb;
      cap_par[2 * c->ncap + m] = h.G;
      cap_par[3 * c->ncap + m] = h.C;
      X.insert(X.end(), h.X0.begin(), h.X0.end());
      for (int l = 0; l < h.nn; ++l) {
        ncap.push_back(m);
        rprev.push_back(noff + (l + h.nn - 1) % h.nn);
        rnext.push_back(noff + (l + 1) % h.nn);
      }
      std::map<std::pair<int, int>, int> edge_tri;
      for (int e = 0; e < h.ne; ++e) {
        ecap.push_back(m);
        for (int q = 0; q < c->NV; ++q) {
          int v = noff + h.E[c->NV * e + q];
          E.push_back(v);
          inc[v].push_back(eoff + e);
        }
        if (c->NV == 2) {
          const double* a = &h.X0[3 * h.E[2 * e]];
          const double* b = &h.X0[3 * h.E[2 * e + 1]];
          ds0.push_back(sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[2] - a[2]) * (b[2] - a[2])));
          A0.push_back(0);
          for (int k = 0; k < 3; ++k) G0i.push_back(0);
        } else {
          const double* a = &h.X0[3 * h.E[3 * e]];
          const double* b = &h.X0[3 * h.E[3 * e + 1]];
          const double* cc = &h.X0[3 * h.E[3 * e + 2]];
          double e1[3], e2[3];
          for (int k = 0; k < 3; ++k) { e1[k] = b[k] - a[k]; e2[k] = cc[k] - a[k]; }
          double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
          double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
          double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
          double det = g11 * g22 - g12 * g12;
          ds0.push_back(0);
          A0.push_back(0.5 * sqrt(det));
          G0i.push_back(g22 / det);
          G0i.push_back(-g12 / det);
          G0i.push_back(g11 / det);
          for (int q = 0; q < 3; ++q) edge_tri[{h.E[3 * e + q], h.E[3 * e + (q + 1) % 3]}] = e;
        }
      }
      for (int e = 0; e < h.ne; ++e)
        for (int q = 0; q < 3; ++q) {
          if (c->NV == 2) { adj.push_back(0); continue; }
          int va = h.E[3 * e + q], vb = h.E[3 * e + (q + 1) % 3];
          auto it = edge_tri.find({vb, va});
          int other = it == edge_tri.end() ? e : it->second;
          adj.push_back(eoff + other);
          if (va < vb) {  // each undirected edge once: vertices, left face, right face
            edges.push_back(noff + va);
            edges.push_back(noff + vb);
            edges.push_back(eoff + e);
            edges.push_back(eoff + other);
          }
        }
      noff += h.nn;
      eoff += h.ne;
    }
    std::vector<int> inc_off(c->nn + 1, 0), incl;
    for (int v = 0; v < c->nn; ++v) {
      std::sort(inc[v].begin(), inc[v].end());
      inc_off[v + 1] = inc_off[v] + (int)inc[v].size();
      incl.insert(incl.end(), inc[v].begin(), inc[v].end());
    }
    // distinct 1-ring neighbours of every node, in the order of its incident
    // elements (ascending) and of their vertices
    std::vector<int> ring_off(c->nn + 1, 0), ring;
    int max_inc = 0, max_ring = 0;
    for (int v = 0; v < c->nn; ++v) {
      const size_t r0 = ring.size();
      for (int e : inc[v])
        for (int q = 0; q < c->NV; ++q) {
          const int u = E[(size_t)c->NV * e + q];
          if (u != v && std::find(ring.begin() + r0, ring.end(), u) == ring.end()) ring.push_back(u);
        }
      ring_off[v + 1] = (int)ring.size();
      max_inc = std::max(max_inc, (int)inc[v].size());
      max_ring = std::max(max_ring, (int)(ring.size() - r0));
    }
    if (c->NV == 3 && (max_inc > 16 || max_ring > 15)) {
      set_error("membrane: a node has more than 16 incident triangles or 15 neighbours");
      delete c;
      return TLB_ERR_ARG;
    }
    auto up = [&](const Region& reg, const void* src, size_t n) {
      return cuda_check(cudaMemcpyAsync(c->base + reg.off, src, n, cudaMemcpyHostToDevice, st), "upload");
    };
    tlb_status u = TLB_OK;
    u = u != TLB_OK ? u : up(c->L.X, X.data(), X.size() * 8);
    u = u != TLB_OK ? u : up(c->L.E, E.data(), E.size() * 4);
    u = u != TLB_OK ? u : up(c->L.ecap, ecap.data(), ecap.size() * 4);
    u = u != TLB_OK ? u : up(c->L.ncap, ncap.data(), ncap.size() * 4);
    u = u != TLB_OK ? u : up(c->L.cap_par, cap_par.data(), cap_par.size() * 8);
    u = u != TLB_OK ? u : up(c->L.ds0, ds0.data(), ds0.size() * 8);
    u = u != TLB_OK ? u : up(c->L.rprev, rprev.data(), rprev.size() * 4);
    u = u != TLB_OK ? u : up(c->L.rnext, rnext.data(), rnext.size() * 4);
    u = u != TLB_OK ? u : up(c->L.A0, A0.data(), A0.size() * 8);
    u = u != TLB_OK ? u : up(c->L.G0i, G0i.data(), G0i.size() * 8);
    // the elastic constants in the working precision (FP32 kernels read
    // them without FP64 conversions)
    {
      std::vector<double> skc(5 * (size_t)c->ne, 0.0);
      if (c->NV == 3)
        for (int t = 0; t < c->ne; ++t) {
          const double* Gi = &G0i[3 * (size_t)t];
          const double k[5] = {Gi[0], 2.0 * Gi[1], Gi[2], Gi[0] * Gi[2] - Gi[1] * Gi[1], A0[t]};
          for (int j = 0; j < 5; ++j) skc[5 * (size_t)t + j] = k[j];
        }
      auto up_real = [&](const Region& reg, const std::vector<double>& v) {
        if (c->ts.real == 8) return up(reg, v.data(), v.size() * 8);
        std::vector<float> f(v.begin(), v.end());
        return up(reg, f.data(), f.size() * 4);
      };
      u = u != TLB_OK ? u : up_real(c->L.skc, skc);
      u = u != TLB_OK ? u : up_real(c->L.capr, cap_par);
    }
    u = u != TLB_OK ? u : up(c->L.inc_off, inc_off.data(), inc_off.size() * 4);
    u = u != TLB_OK ? u : up(c->L.inc, incl.data(), incl.size() * 4);
    u = u != TLB_OK ? u : up(c->L.adj, adj.data(), adj.size() * 4);
    u = u != TLB_OK ? u : up(c->L.ring_off, ring_off.data(), ring_off.size() * 4);
    if (!ring.empty()) u = u != TLB_OK ? u : up(c->L.ring, ring.data(), ring.size() * 4);
    if ((int)edges.size() != 4 * c->nedge) {
      set_error("membrane is not a closed surface (every edge must belong to two triangles)");
      delete c;
      return TLB_ERR_ARG;
    }
    if (!edges.empty()) u = u != TLB_OK ? u : up(c->L.edges, edges.data(), edges.size() * 4);
    if (u == TLB_OK) u = cuda_check(cudaStreamSynchronize(st), "upload sync");
    if (u != TLB_OK) { delete c; return u; }
  }
  r = cuda_check(cudaStreamSynchronize(st), "create");
  if (r != TLB_OK) { delete c; return r; }
  *ctx_out = c;
  return TLB_OK;
}

tlb_status tlb_init_fields(void* ctx, const double* C, const double* u) {
  Ctx* c = (Ctx*)ctx;
  if (!c) { set_error("ctx is NULL"); return TLB_ERR_ARG; }
  return c->impl->init_fields(c, C, u);
}

tlb_status tlb_step(void* ctx, long n_steps) {
  Ctx* c = (Ctx*)ctx;
  if (!c) { set_error("ctx is NULL"); return TLB_ERR_ARG; }
  if (!c->initialised) { set_error("tlb_step before tlb_init_fields"); return TLB_ERR_STATE; }
  if (n_steps < 0) { set_error("n_steps < 0"); return TLB_ERR_ARG; }
  c->launches = 0;
  return c->impl->step(c, n_steps);
}

tlb_status tlb_read_field(void* ctx, int field, double* dst, size_t n_values) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !dst) { set_error("ctx/dst is NULL"); return TLB_ERR_ARG; }
  return c->impl->read_field(c, field, dst, n_values);
}

tlb_status tlb_read_nodes(void* ctx, int capsule, double* dst, size_t n_values) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !dst) { set_error("ctx/dst is NULL"); return TLB_ERR_ARG; }
  if (capsule < 0 || capsule >= c->ncap) { set_error("no such capsule"); return TLB_ERR_ARG; }
  int off = 0;
  for (int m = 0; m < capsule; ++m) off += c->mems[m].nn;
  const int nn = c->mems[capsule].nn;
  if (n_values < (size_t)3 * nn) { set_error("read_nodes: buffer too small"); return TLB_ERR_ARG; }
  std::vector<double> h(3 * nn);
  TLB_CUDA(cudaMemcpyAsync(h.data(), c->ptr<double>(c->L.X) + 3 * off, 3 * nn * 8, cudaMemcpyDeviceToHost, c->stream));
  TLB_CUDA(cudaStreamSynchronize(c->stream));
  for (int l = 0; l < nn; ++l) {
    if (c->p.dim == 2) {
      dst[3 * l] = h[3 * l];
      dst[3 * l + 1] = h[3 * l + 2];
      dst[3 * l + 2] = 0.0;
    } else {
      for (int k = 0; k < 3; ++k) dst[3 * l + k] = h[3 * l + k];
    }
  }
  return TLB_OK;
}

tlb_status tlb_write_nodes(void* ctx, int capsule, const double* src, size_t n_values) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !src) { set_error("ctx/src is NULL"); return TLB_ERR_ARG; }
  if (capsule < 0 || capsule >= c->ncap) { set_error("no such capsule"); return TLB_ERR_ARG; }
  int off = 0;
  for (int m = 0; m < capsule; ++m) off += c->mems[m].nn;
  const int nn = c->mems[capsule].nn;
  if (n_values < (size_t)3 * nn) { set_error("write_nodes: buffer too small"); return TLB_ERR_ARG; }
  std::vector<double> h(3 * nn);
  for (int l = 0; l < nn; ++l) {
    if (c->p.dim == 2) {
      h[3 * l] = src[3 * l];
      h[3 * l + 1] = 0.0;
      h[3 * l + 2] = src[3 * l + 1];
    } else {
      for (int k = 0; k < 3; ++k) h[3 * l + k] = src[3 * l + k];
    }
  }
  TLB_CUDA(cudaMemcpyAsync(c->ptr<double>(c->L.X) + 3 * off, h.data(), 3 * nn * 8, cudaMemcpyHostToDevice, c->stream));
  TLB_CUDA(cudaStreamSynchronize(c->stream));
  c->box_stale = true;
  return TLB_OK;
}

tlb_status tlb_read_populations(void* ctx, double* dst, size_t n_values) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !dst) { set_error("ctx/dst is NULL"); return TLB_ERR_ARG; }
  if (n_values < (size_t)3 * c->Q * c->N) { set_error("read_populations: buffer too small"); return TLB_ERR_ARG; }
  return c->impl->read_pops(c, dst);
}

tlb_status tlb_write_populations(void* ctx, const double* src, size_t n_values) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !src) { set_error("ctx/src is NULL"); return TLB_ERR_ARG; }
  if (n_values < (size_t)3 * c->Q * c->N) { set_error("write_populations: buffer too small"); return TLB_ERR_ARG; }
  return c->impl->write_pops(c, src);
}

tlb_status tlb_diagnostics(void* ctx, tlb_diag* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !out) { set_error("ctx/out is NULL"); return TLB_ERR_ARG; }
  return c->impl->diagnostics(c, out);
}

tlb_status tlb_contact_angle(void* ctx, double* out, size_t n_values) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !out) { set_error("ctx/out is NULL"); return TLB_ERR_ARG; }
  if (n_values < 4 * (size_t)c->ncap) { set_error("contact_angle: out holds fewer than 4 values per capsule"); return TLB_ERR_ARG; }
  if (!c->initialised) { set_error("contact_angle: context not initialised"); return TLB_ERR_STATE; }
  return c->impl->contact_angle(c, out);
}

// Residual values from the maxima the residual kernel folded into res[0..2].
static void residual_values(const unsigned long long* bits, long dt, double* out) {
  double m = 0;
  for (int q = 0; q < 3; ++q) {
    double v;
    memcpy(&v, &bits[q], sizeof(double));
    out[q] = v;
    m = std::max(m, v);
  }
  out[3] = dt > 0 ? m / (double)dt : 0.0;
}

tlb_status tlb_residual(void* ctx, double* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !out) { set_error("ctx/out is NULL"); return TLB_ERR_ARG; }
  if (!c->initialised) { set_error("tlb_residual before tlb_init_fields"); return TLB_ERR_STATE; }
  tlb_status s = c->impl->residual_launch(c);
  if (s != TLB_OK) return s;
  unsigned long long h[4];
  TLB_CUDA(cudaMemcpyAsync(h, c->ptr<unsigned long long>(c->L.res), sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  TLB_CUDA(cudaStreamSynchronize(c->stream));
  residual_values(h, c->t - c->t_snap, out);
  c->t_snap = c->t;
  return TLB_OK;
}

tlb_status tlb_profile_steps(void* ctx, long n_steps, tlb_profile* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !out) { set_error("ctx/out is NULL"); return TLB_ERR_ARG; }
  if (!c->initialised) { set_error("tlb_profile_steps before tlb_init_fields"); return TLB_ERR_STATE; }
  PhaseEvents pe;
  for (int k = 0; k < 5; ++k) TLB_CUDA(cudaEventCreate(&pe.ev[k]));
  c->prof = &pe;
  for (int k = 0; k < 4; ++k) c->prof_ms[k] = 0;
  c->launches = 0;
  tlb_status s = c->impl->step(c, n_steps);
  c->prof = nullptr;
  for (int k = 0; k < 5; ++k) cudaEventDestroy(pe.ev[k]);
  if (s != TLB_OK) return s;
  out->steps = n_steps;
  out->ms_moments = c->prof_ms[0];
  out->ms_ibm = c->prof_ms[1];
  out->ms_collide = c->prof_ms[2];
  out->ms_interp = c->prof_ms[3];
  out->launches_per_step = n_steps > 0 ? c->launches / n_steps : 0;
  return TLB_OK;
}

tlb_status tlb_autotune(void* ctx, int* tile_variant, int* z_chunk) {
  Ctx* c = (Ctx*)ctx;
  if (!c) { set_error("ctx is NULL"); return TLB_ERR_ARG; }
  if (!c->initialised) { set_error("tlb_autotune before tlb_init_fields"); return TLB_ERR_STATE; }
  return c->impl->autotune(c, tile_variant, z_chunk);
}

tlb_status tlb_set_tile(void* ctx, int tile_variant, int z_chunk) {
  Ctx* c = (Ctx*)ctx;
  if (!c) { set_error("ctx is NULL"); return TLB_ERR_ARG; }
  if (tile_variant < 0 || tile_variant >= COLLIDE_NVAR || z_chunk < 1 || z_chunk > c->nz) {
    set_error("set_tile: tile_variant must be 0..31 and z_chunk 1..nz");
    return TLB_ERR_ARG;
  }
  if (!c->variant_ok(tile_variant)) {
    set_error("set_tile: variants 13..18 need tau = tau_phi = tau_psi = 1, TLB_FORCE_EDM and the potential "
              "force (and are the only ones with moment storage); 19..21 are those of the pressure-tensor force");
    return TLB_ERR_ARG;
  }
  c->tile_variant = tile_variant;
  c->tiles_zc = z_chunk;
  return TLB_OK;
}

tlb_status tlb_set_graphs(void* ctx, int on) {
  Ctx* c = (Ctx*)ctx;
  if (!c) { set_error("ctx is NULL"); return TLB_ERR_ARG; }
  if (!on) {
    TLB_CUDA(cudaStreamSynchronize(c->stream));
    c->drop_graphs();
  }
  c->graphs = on != 0;
  return TLB_OK;
}

long tlb_last_launch_count(void* ctx) {
  Ctx* c = (Ctx*)ctx;
  return c ? c->launches : 0;
}

void tlb_destroy(void* ctx) { delete (Ctx*)ctx; }

}  // extern "C"
