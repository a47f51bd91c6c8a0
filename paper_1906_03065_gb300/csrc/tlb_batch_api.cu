// C ABI of the batched sweep (see include/tlb.h): sub-arena planning,
// instance creation, activity and the run-to-residual loop.  The kernels
// and the per-type driver are in tlb_batch.cuh.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tlb_ctx.h"

static size_t align256b(size_t v) { return (v + 255) & ~(size_t)255; }

// Arena plan of a batch: instance sub-arenas in order, then the argument
// tables (two parities), the virtual-grid tables and the residual slots.
struct BatchPlan {
  std::vector<size_t> off, bytes;
  size_t targs[2], vg, res, total;
};

static tlb_status batch_plan(const tlb_instance_desc* inst, int n, BatchPlan& bp) {
  if (!inst || n <= 0) { set_error("batch: inst is NULL or n_inst <= 0"); return TLB_ERR_ARG; }
  if (n > 4096) { set_error("batch: at most 4096 instances"); return TLB_ERR_ARG; }
  size_t off = 0;
  bp.off.resize(n);
  bp.bytes.resize(n);
  for (int i = 0; i < n; ++i) {
    if (inst[i].params.dim != inst[0].params.dim || inst[i].params.storage != inst[0].params.storage) {
      set_error("batch: every instance must have the same dim and storage");
      return TLB_ERR_ARG;
    }
    size_t b = 0;
    tlb_status s = tlb_state_bytes(&inst[i].params, inst[i].mems, inst[i].n_mem, &b);
    if (s != TLB_OK) {
      set_error("batch instance " + std::to_string(i) + ": " + tlb_last_error());
      return s;
    }
    bp.off[i] = off;
    bp.bytes[i] = b;
    off = align256b(off + b);
  }
  for (int q = 0; q < 2; ++q) {
    bp.targs[q] = off;
    off = align256b(off + (size_t)n * Batch::ARGS_BYTES);
  }
  bp.vg = off;
  off = align256b(off + (size_t)Batch::NPH * Batch::MAXOPS * n * 16);
  bp.res = off;
  off = align256b(off + (size_t)n * 4 * 8);
  bp.total = off;
  return TLB_OK;
}

// Virtual blocks of the box-sized operations (profile band, spreading): the
// work scales with the marker box, estimated from the initial markers.
static void box_estimates(const Ctx* c, int* band_blocks, int* spread_blocks) {
  if (c->nn == 0) { *band_blocks = *spread_blocks = 0; return; }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (const HostMem& m : c->mems)
    for (int l = 0; l < m.nn; ++l)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], m.X0[3 * l + d]);
        hi[d] = std::max(hi[d], m.X0[3 * l + d]);
      }
  const int n[3] = {c->nx, c->ny, c->nz};
  const double margin = 2.0 * (ceil(c->p.dc) + 2.0) + 2.0;
  double cells = 1, bricks = 1;
  for (int d = 0; d < 3; ++d) {
    cells *= std::min((double)n[d], hi[d] - lo[d] + margin);
    bricks *= std::min(ceil(n[d] / 4.0), ceil((hi[d] - lo[d] + 4.0) / 4.0) + 1.0);
  }
  // about two box cells per thread of a 128-thread block
  *band_blocks = (int)std::max(1.0, std::min(65536.0, ceil(cells / 256.0)));
  *spread_blocks = (int)std::max(1.0, std::min((double)c->nbricks, bricks));
}

extern "C" {

tlb_status tlb_batch_state_bytes(const tlb_instance_desc* inst, int n_inst, size_t* bytes) {
  if (!bytes) { set_error("bytes is NULL"); return TLB_ERR_ARG; }
  BatchPlan bp;
  tlb_status s = batch_plan(inst, n_inst, bp);
  if (s != TLB_OK) return s;
  *bytes = bp.total;
  return TLB_OK;
}

tlb_status tlb_batch_create(const tlb_instance_desc* inst, int n_inst, void* arena, size_t bytes, void* cuda_stream,
                            void** batch_out) {
  if (!arena || !batch_out) { set_error("arena and batch_out must be non-NULL"); return TLB_ERR_ARG; }
  if (((uintptr_t)arena) & 255) { set_error("arena must be 256-byte aligned"); return TLB_ERR_ARG; }
  BatchPlan bp;
  tlb_status s = batch_plan(inst, n_inst, bp);
  if (s != TLB_OK) return s;
  if (bytes < bp.total) {
    set_error("batch arena too small: need " + std::to_string(bp.total) + " bytes");
    return TLB_ERR_ALLOC;
  }
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].params.state != TLB_STATE_POPULATIONS) {
      set_error("batch: instances keep populations (TLB_STATE_POPULATIONS)");
      return TLB_ERR_ARG;
    }
  Batch* b = new Batch();
  b->dim = inst[0].params.dim;
  b->storage = inst[0].params.storage;
  b->stream = (cudaStream_t)cuda_stream;
  b->base = (char*)arena;
  b->bytes = bytes;
  switch (b->dim * 10 + b->storage) {
    case 20: b->impl = make_batch_impl_d2q9_f64(); break;
    case 21: b->impl = make_batch_impl_d2q9_f32(); break;
    case 31: b->impl = make_batch_impl_d3q19_f32(); break;
    case 32: b->impl = make_batch_impl_d3q19_f16(); break;
    case 33: b->impl = make_batch_impl_d3q19_bf16(); break;
    default: set_error("batch: unsupported dim/storage"); delete b; return TLB_ERR_ARG;
  }
  s = cuda_check(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "batch capture stream");
  if (s != TLB_OK) { delete b; return s; }
  int nzmax = 1;
  for (int i = 0; i < n_inst; ++i) {
    void* h = nullptr;
    s = tlb_create(&inst[i].params, inst[i].mems, inst[i].n_mem, b->base + bp.off[i], bp.bytes[i], cuda_stream, &h);
    if (s != TLB_OK) {
      set_error("batch instance " + std::to_string(i) + ": " + tlb_last_error());
      delete b;
      return s;
    }
    Ctx* c = (Ctx*)h;
    b->inst.push_back(c);
    b->act.push_back(i);
    int bb = 0, sb = 0;
    box_estimates(c, &bb, &sb);
    b->band_blocks.push_back(bb);
    b->spread_blocks.push_back(sb);
    nzmax = std::max(nzmax, c->nz);
  }
  b->zc = nzmax >= 64 ? 16 : std::min(nzmax, 8);
  // the tau = 1 collide wherever it applies; one force form per batch
  b->tile_variant = 0;
  for (int v : {13, 19, 0}) {
    bool ok = true;
    for (Ctx* c : b->inst) ok = ok && c->variant_ok(v);
    if (ok) {
      b->tile_variant = v;
      break;
    }
  }
  for (Ctx* c : b->inst)
    if (!c->variant_ok(b->tile_variant)) {
      set_error("batch: instances mix force forms");
      delete b;
      return TLB_ERR_ARG;
    }
  for (int q = 0; q < 2; ++q) b->targs[q] = {bp.targs[q], (size_t)n_inst * Batch::ARGS_BYTES};
  b->vg = {bp.vg, (size_t)Batch::NPH * Batch::MAXOPS * n_inst * 16};
  b->res = {bp.res, (size_t)n_inst * 4 * 8};
  *batch_out = b;
  return TLB_OK;
}

tlb_status tlb_batch_instance(void* batch, int i, void** ctx_out) {
  Batch* b = (Batch*)batch;
  if (!b || !ctx_out) { set_error("batch/ctx_out is NULL"); return TLB_ERR_ARG; }
  if (i < 0 || i >= (int)b->inst.size()) { set_error("batch: instance index out of range"); return TLB_ERR_ARG; }
  *ctx_out = b->inst[i];
  return TLB_OK;
}

tlb_status tlb_batch_set_active(void* batch, const int* flags) {
  Batch* b = (Batch*)batch;
  if (!b || !flags) { set_error("batch/flags is NULL"); return TLB_ERR_ARG; }
  std::vector<int> act;
  for (int i = 0; i < (int)b->inst.size(); ++i)
    if (flags[i]) act.push_back(i);
  if (act != b->act) {
    b->act = act;
    b->graph_dirty = true;
  }
  return TLB_OK;
}

static tlb_status check_initialised(Batch* b) {
  for (int i : b->act)
    if (!b->inst[i]->initialised) {
      set_error("batch: instance " + std::to_string(i) + " is not initialised");
      return TLB_ERR_STATE;
    }
  return TLB_OK;
}

tlb_status tlb_batch_step(void* batch, long n_steps) {
  Batch* b = (Batch*)batch;
  if (!b) { set_error("batch is NULL"); return TLB_ERR_ARG; }
  if (n_steps < 0) { set_error("n_steps < 0"); return TLB_ERR_ARG; }
  tlb_status s = check_initialised(b);
  if (s != TLB_OK) return s;
  b->launches = 0;
  return b->impl->step(b, n_steps);
}

tlb_status tlb_batch_run(void* batch, long max_steps, long check_every, double tol, long* steps_done,
                         double* residual) {
  Batch* b = (Batch*)batch;
  if (!b) { set_error("batch is NULL"); return TLB_ERR_ARG; }
  if (max_steps < 0 || check_every <= 0) { set_error("batch_run: max_steps < 0 or check_every <= 0"); return TLB_ERR_ARG; }
  tlb_status s = check_initialised(b);
  if (s != TLB_OK) return s;
  b->launches = 0;
  const int n = (int)b->inst.size();
  std::vector<double> last(n, NAN);
  std::vector<unsigned long long> h((size_t)4 * n);
  long done = 0;
  while (!b->act.empty() && done < max_steps) {
    const long k = std::min(check_every, max_steps - done);
    s = b->impl->step(b, k);
    if (s != TLB_OK) return s;
    s = b->impl->residual(b);
    if (s != TLB_OK) return s;
    TLB_CUDA(cudaMemcpyAsync(h.data(), b->ptr<unsigned long long>(b->res), h.size() * 8, cudaMemcpyDeviceToHost,
                             b->stream));
    TLB_CUDA(cudaStreamSynchronize(b->stream));
    std::vector<int> still;
    for (int i : b->act) {
      Ctx* c = b->inst[i];
      double m = 0;
      for (int q = 0; q < 3; ++q) {
        double v;
        memcpy(&v, &h[4 * (size_t)i + q], sizeof(double));
        m = std::max(m, v);
      }
      const long dt = c->t - c->t_snap;
      c->t_snap = c->t;
      last[i] = dt > 0 ? m / (double)dt : 0.0;
      if (!(last[i] <= tol)) still.push_back(i);
    }
    if (still != b->act) {
      b->act = still;
      b->graph_dirty = true;
    }
    done += k;
  }
  for (int i = 0; i < n; ++i) {
    if (steps_done) steps_done[i] = b->inst[i]->t;
    if (residual) residual[i] = last[i];
  }
  return TLB_OK;
}

tlb_status tlb_batch_autotune(void* batch, int* tile_variant, int* z_chunk) {
  Batch* b = (Batch*)batch;
  if (!b) { set_error("batch is NULL"); return TLB_ERR_ARG; }
  tlb_status s = check_initialised(b);
  if (s != TLB_OK) return s;
  return b->impl->autotune(b, tile_variant, z_chunk);
}

tlb_status tlb_batch_profile_steps(void* batch, long n_steps, double* ms_per_phase) {
  Batch* b = (Batch*)batch;
  if (!b || !ms_per_phase) { set_error("batch/ms_per_phase is NULL"); return TLB_ERR_ARG; }
  if (n_steps < 0) { set_error("n_steps < 0"); return TLB_ERR_ARG; }
  tlb_status s = check_initialised(b);
  if (s != TLB_OK) return s;
  b->launches = 0;
  return b->impl->profile(b, n_steps, ms_per_phase);
}

long tlb_batch_launch_count(void* batch) {
  Batch* b = (Batch*)batch;
  return b ? b->launches : 0;
}

void tlb_batch_destroy(void* batch) { delete (Batch*)batch; }

}  // extern "C"
