// Checkpoint and resume of a context (tlb_save / tlb_load) and the
// single-context run to a residual tolerance (tlb_run); see include/tlb.h.
//
// A checkpoint holds exactly the state a continued run reads: the current
// population buffer (populations are stored post-collision), the profile I
// (cells that leave the moving marker box keep their last value), the
// marker positions, the residual's reference state and the step counters.
// Everything else is rebuilt within the next step: moments, potentials,
// forces, keys, bricks; the marker box is recomputed from the markers, which
// gives the same integers as the accumulator the advection leaves.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "tlb_ctx.h"

namespace {

constexpr char kMagic[8] = {'T', 'L', 'B', 'C', 'K', 'P', 'T', '1'};
constexpr int kSections = 6;

struct Header {
  char magic[8];
  uint32_t version, header_bytes;
  // the parameters, field by field (no struct padding in the file)
  int32_t dim, nx, ny, nz, wall_last, storage, forcing, state, force_form, pad;
  double tau, tau_phi, tau_psi, gamma_phi, gamma_psi, alpha, kappa[3], kappa_c, dc, u0[3], interface_pos;
  int64_t nn, ne, N, P, t, t_snap;
  uint64_t mem_hash;  // the membranes: reference shapes, elements, moduli
  uint64_t sec_bytes[kSections];
};

// FNV-1a over the membrane descriptors the context was created with, so a
// checkpoint only loads onto a context with the same membranes (shape,
// connectivity and stiffness), not just the same counts.
uint64_t membrane_hash(const Ctx* c) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  for (const HostMem& m : c->mems) {
    mix(&m.kind, sizeof(m.kind));
    mix(&m.nn, sizeof(m.nn));
    mix(&m.ne, sizeof(m.ne));
    mix(m.X0.data(), m.X0.size() * sizeof(double));
    mix(m.E.data(), m.E.size() * sizeof(int));
    const double mod[4] = {m.ks, m.kb, m.G, m.C};
    mix(mod, sizeof(mod));
  }
  return h;
}

void fill_params(Header& h, const tlb_params& p) {
  h.dim = p.dim;
  h.nx = p.nx;
  h.ny = p.ny;
  h.nz = p.nz;
  h.wall_last = p.wall_last;
  h.storage = p.storage;
  h.forcing = p.forcing;
  h.state = p.state;
  h.force_form = p.force_form;
  h.pad = 0;
  h.tau = p.tau;
  h.tau_phi = p.tau_phi;
  h.tau_psi = p.tau_psi;
  h.gamma_phi = p.gamma_phi;
  h.gamma_psi = p.gamma_psi;
  h.alpha = p.alpha;
  for (int k = 0; k < 3; ++k) h.kappa[k] = p.kappa[k];
  h.kappa_c = p.kappa_c;
  h.dc = p.dc;
  for (int k = 0; k < 3; ++k) h.u0[k] = p.u0[k];
  h.interface_pos = p.interface_pos;
}

bool same_params(const Header& a, const Header& b) {
  if (a.dim != b.dim || a.nx != b.nx || a.ny != b.ny || a.nz != b.nz || a.wall_last != b.wall_last ||
      a.storage != b.storage || a.forcing != b.forcing || a.state != b.state || a.force_form != b.force_form)
    return false;
  const double x[] = {a.tau, a.tau_phi, a.tau_psi, a.gamma_phi, a.gamma_psi, a.alpha, a.kappa[0], a.kappa[1],
                      a.kappa[2], a.kappa_c, a.dc, a.u0[0], a.u0[1], a.u0[2], a.interface_pos};
  const double y[] = {b.tau, b.tau_phi, b.tau_psi, b.gamma_phi, b.gamma_psi, b.alpha, b.kappa[0], b.kappa[1],
                      b.kappa[2], b.kappa_c, b.dc, b.u0[0], b.u0[1], b.u0[2], b.interface_pos};
  return memcmp(x, y, sizeof(x)) == 0;
}

// device regions of the sections, in file order
void sections(Ctx* c, int cur, char** ptr, size_t* bytes) {
  const Region* r[kSections] = {&c->L.lo[cur], &c->L.rest[cur], &c->L.I, &c->L.X, &c->L.snap, &c->L.xsnap};
  for (int k = 0; k < kSections; ++k) {
    ptr[k] = c->base + r[k]->off;
    bytes[k] = r[k]->bytes;
  }
}

Header header_of(Ctx* c, const size_t* bytes) {
  Header h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMagic, 8);
  h.version = 2;
  h.header_bytes = sizeof(Header);
  fill_params(h, c->p);
  h.nn = c->nn;
  h.ne = c->ne;
  h.N = c->N;
  h.P = c->P;
  h.t = c->t;
  h.t_snap = c->t_snap;
  h.mem_hash = membrane_hash(c);
  for (int k = 0; k < kSections; ++k) h.sec_bytes[k] = bytes[k];
  return h;
}

}  // namespace

extern "C" {

tlb_status tlb_save(void* ctx, void* host_blob, size_t* bytes) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !bytes) { set_error("ctx/bytes is NULL"); return TLB_ERR_ARG; }
  if (!c->initialised) { set_error("tlb_save before tlb_init_fields"); return TLB_ERR_STATE; }
  // moment storage: the checkpoint holds the populations the moments stand
  // for (the same values the next pull would rebuild)
  if (tlb_status st = c->impl->sync_pops(c); st != TLB_OK) return st;
  char* dev[kSections];
  size_t sz[kSections];
  sections(c, c->cur, dev, sz);
  size_t total = sizeof(Header);
  for (int k = 0; k < kSections; ++k) total += sz[k];
  if (!host_blob) {
    *bytes = total;
    return TLB_OK;
  }
  if (*bytes < total) {
    set_error("tlb_save: blob too small, need " + std::to_string(total) + " bytes");
    return TLB_ERR_ARG;
  }
  Header h = header_of(c, sz);
  char* out = (char*)host_blob;
  memcpy(out, &h, sizeof(h));
  size_t off = sizeof(h);
  for (int k = 0; k < kSections; ++k) {
    if (sz[k]) TLB_CUDA(cudaMemcpyAsync(out + off, dev[k], sz[k], cudaMemcpyDeviceToHost, c->stream));
    off += sz[k];
  }
  TLB_CUDA(cudaStreamSynchronize(c->stream));
  *bytes = total;
  return TLB_OK;
}

tlb_status tlb_load(void* ctx, const void* host_blob, size_t bytes) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !host_blob) { set_error("ctx/host_blob is NULL"); return TLB_ERR_ARG; }
  if (bytes < sizeof(Header)) { set_error("tlb_load: blob shorter than its header"); return TLB_ERR_ARG; }
  Header h;
  memcpy(&h, host_blob, sizeof(h));
  if (memcmp(h.magic, kMagic, 8) != 0 || h.version != 2 || h.header_bytes != sizeof(Header)) {
    set_error("tlb_load: not a checkpoint of this library version");
    return TLB_ERR_ARG;
  }
  char* dev[kSections];
  size_t sz[kSections];
  sections(c, 0, dev, sz);
  Header mine = header_of(c, sz);
  if (!same_params(h, mine) || h.nn != mine.nn || h.ne != mine.ne || h.N != mine.N || h.P != mine.P ||
      h.mem_hash != mine.mem_hash) {
    set_error("tlb_load: the checkpoint was taken of a context with other parameters or membranes");
    return TLB_ERR_ARG;
  }
  size_t total = sizeof(Header);
  for (int k = 0; k < kSections; ++k) {
    if (h.sec_bytes[k] != sz[k]) { set_error("tlb_load: section sizes differ"); return TLB_ERR_ARG; }
    total += sz[k];
  }
  if (bytes < total) { set_error("tlb_load: blob truncated"); return TLB_ERR_ARG; }
  const char* in = (const char*)host_blob;
  size_t off = sizeof(Header);
  for (int k = 0; k < kSections; ++k) {
    if (sz[k]) TLB_CUDA(cudaMemcpyAsync(dev[k], in + off, sz[k], cudaMemcpyHostToDevice, c->stream));
    off += sz[k];
  }
  TLB_CUDA(cudaMemsetAsync(c->ptr<char>(c->L.status), 0, c->L.status.bytes, c->stream));
  TLB_CUDA(cudaStreamSynchronize(c->stream));
  c->cur = 0;
  c->t = h.t;
  c->t_snap = h.t_snap;
  c->initialised = true;
  c->box_stale = true;
  c->state_in_pops = true;  // (moment storage: the next step pulls them)
  c->pops_stale = false;
  return TLB_OK;
}

tlb_status tlb_run(void* ctx, long max_steps, long check_every, double tol, long* steps_done, double* residual) {
  Ctx* c = (Ctx*)ctx;
  if (!c) { set_error("ctx is NULL"); return TLB_ERR_ARG; }
  if (max_steps < 0 || check_every <= 0) { set_error("tlb_run: max_steps < 0 or check_every <= 0"); return TLB_ERR_ARG; }
  double r[4] = {0, 0, 0, NAN};
  long done = 0;
  while (done < max_steps) {
    const long k = std::min(check_every, max_steps - done);
    tlb_status s = tlb_step(ctx, k);
    if (s == TLB_OK) s = tlb_residual(ctx, r);
    if (s != TLB_OK) return s;
    done += k;
    if (r[3] <= tol) break;
  }
  if (steps_done) *steps_done = c->t;
  if (residual) *residual = r[3];
  return TLB_OK;
}

}  // extern "C"
