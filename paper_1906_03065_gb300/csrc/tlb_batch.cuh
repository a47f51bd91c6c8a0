// Batched sweep: many independent lattices (a parameter sweep with uneven
// sizes and membranes) advanced together.  Each phase of the step is ONE
// persistent launch: its CTAs walk the concatenated virtual grids of every
// (kernel body, instance) pair of the phase, so small instances do not leave
// the GPU idle and the step costs six launches however many instances run.
// Two steps are captured in one CUDA graph.  The bodies are the ones the
// single-lattice kernels run, so a batched instance evolves as it would
// alone (the same bits in FP64; FP32 code may differ in the last place where
// the compiler fuses multiply-adds differently in the combined kernels).
#pragma once
#include <algorithm>
#include <vector>

#include "tlb_impl.cuh"

// Everything the kernels of one instance read, for one parity of its
// population buffers.
template <int MODE>
struct BArgs {
  LBArgs<MODE> lb;
  IBArgs<typename Prec<MODE>::Real> ib;
  ResPtrs rp;
};

// Start-of-step membrane bookkeeping that the single-lattice path does with
// memsets and a copy: clear the coupling sums and the brick counters, take
// the snapshot of the marker box and reset its accumulator.
template <int MODE>
__device__ __forceinline__ void pre_body(const BArgs<MODE>& s, const Blk& blk) {
  const auto& a = s.ib;
  const long long n = 3ll * a.nn;
  for (long long i = (long long)blk.x * blockDim.x + threadIdx.x; i < n; i += (long long)blk.gx * blockDim.x)
    a.ncpl[i] = 0;
  if (blk.x == 0 && threadIdx.x < 6) {
    a.box[6 + threadIdx.x] = a.box[threadIdx.x];
    a.box[threadIdx.x] = 0x7F7F7F7F;
  }
  if (blk.x == 0 && threadIdx.x < 2) a.ctr[threadIdx.x] = 0;
}

// Operations: one kernel body applied to one virtual block of one instance.
template <int MODE> struct OpPre {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { pre_body<MODE>(s, b); }
};
template <class L, int MODE> struct OpMoments {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { moments_body<L, MODE>(s.lb, b); }
};
template <int MODE> struct OpGeometry {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { geometry_body(s.ib, b); }
};
template <int MODE> struct OpBrickCount {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { brick_count_body(s.ib, b); }
};
template <int MODE> struct OpNodeForces {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { node_forces_body(s.ib, b); }
};
template <int MODE> struct OpScatter {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { dist_scatter_body(s.ib, b); }
};
template <int MODE> struct OpBrickCompact {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { brick_compact_body(s.ib, b); }
};
template <int MODE> struct OpBand {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { band_body(s.ib, b); }
};
template <int MODE> struct OpBrickFill {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { brick_fill_body(s.ib, b); }
};
template <int MODE> struct OpFill {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { fill_body(s.ib, b); }
};
template <int MODE> struct OpSpread {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) { spread_body(s.ib, b); }
};
template <class L, int MODE, int TX, int TY, int FORM> struct OpCollide {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) {
    collide_body<L, MODE, TX, TY, FORM>(s.lb, b);
  }
};
template <class L, int MODE> struct OpInterp {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) {
    interp_advect_body<L, MODE>(s.ib, s.lb.lo_dst, b);
  }
};
template <class L, int MODE> struct OpResidual {
  static __device__ __forceinline__ void run(const BArgs<MODE>& s, const Blk& b) {
    residual_body<L, MODE>(s.lb.G, s.lb.lo_src, s.lb.rest_src, s.ib.X, s.ib.nn, s.rp, b);
  }
};

template <class BA, class Op, class... Rest>
__device__ __forceinline__ void run_op(int k, const BA& a, const Blk& b) {
  if (k == 0) {
    Op::run(a, b);
  } else {
    if constexpr (sizeof...(Rest) > 0) run_op<BA, Rest...>(k - 1, a, b);
  }
}

// One phase of the batched step.  Entry e = op * n_inst + instance of the
// table `vg` holds that pair's virtual grid (x, y, z) and its first virtual
// block (w); entries are in order of first block.  CTAs take virtual blocks
// round-robin and find their entry by binary search.
template <int NT, int MINB, class BA, class... Ops>
__global__ void __launch_bounds__(NT, MINB) k_phase(const BA* __restrict__ args, const int4* __restrict__ vg,
                                                    int n_inst, int n_ent, int total) {
  for (int v = blockIdx.x; v < total; v += gridDim.x) {
    int lo = 0, hi = n_ent - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (vg[mid].w <= v) lo = mid;
      else hi = mid - 1;
    }
    const int4 g = vg[lo];
    const int r = v - g.w;
    const Blk b = {r % g.x, (r / g.x) % g.y, r / (g.x * g.y), g.x, g.y, g.z};
    run_op<BA, Ops...>(lo / n_inst, args[lo % n_inst], b);
    __syncthreads();  // the next virtual block reuses the shared memory
  }
}

// Host driver of a batch of one lattice type and storage.
template <class L, int MODE>
struct BatchImpl : BatchBase {
  using Real = typename Prec<MODE>::Real;
  using Store = typename Prec<MODE>::Store;
  using Rest = typename Prec<MODE>::Rest;
  using BA = BArgs<MODE>;
  using I = Impl<L, MODE>;
  static constexpr int NT = 128;  // threads of every phase except the collide

  enum Op { PRE, MOM, GEOM, BCOUNT, NODEF, SCAT, BCOMP, BAND, BFILL, FILL, SPREAD, COLL, INTERP, RESID };
  // ops of each phase, in the order of the phase kernel's template list
  static std::vector<int> phase_ops(int ph) {
    switch (ph) {
      case 0: return {PRE, MOM, GEOM, BCOUNT};  // depend on X(t) and the populations only
      case 1: return {NODEF, SCAT, BCOMP};      // need the normals and the brick counts
      case 2: return {BAND, BFILL};             // need the keys, psi(t) and the brick offsets
      case 3: return {SPREAD, FILL};            // need the band and the coupling sums
      case 4: return {COLL};
      case 5: return {INTERP};
      default: return {RESID};
    }
  }

  static unsigned cdiv(long long n, long long d) { return (unsigned)((n + d - 1) / d); }

  // virtual grid of one op for instance c
  static int3 op_grid(const Batch* b, int i, int op) {
    const Ctx* c = b->inst[i];
    const bool mem = c->nn > 0;
    switch (op) {
      case PRE: return {mem ? (int)std::min<unsigned>(64, std::max(1u, cdiv(3ll * c->nn, NT))) : 0, 1, 1};
      case MOM: return {(int)cdiv(c->N, NT), 1, 1};
      case GEOM: return {mem ? (int)cdiv((long long)c->ne + c->nn, NT) : 0, 1, 1};
      case BCOUNT: return {mem ? (int)cdiv(c->nn, NT) : 0, 1, 1};
      case NODEF: return {mem ? (int)cdiv(32ll * c->nn, NT) : 0, 1, 1};
      case SCAT: {
        const long long nfeat = (long long)c->ne + (c->NV == 3 ? c->nedge : 0) + c->nn;
        return {mem ? SCAT_SPLIT * (int)cdiv(nfeat, 32 * scatter_warps<typename Prec<MODE>::Real>()) : 0, 1, 1};
      }
      case BCOMP: return {mem ? (int)cdiv(c->nbricks, NT) : 0, 1, 1};
      case BAND: return {mem ? b->band_blocks[i] : 0, 1, 1};
      case BFILL: return {mem ? (int)cdiv(c->nn, NT) : 0, 1, 1};
      case FILL: return {mem ? (int)cdiv(32ll * c->nx * c->ny, NT) : 0, 1, 1};
      case SPREAD: return {mem ? b->spread_blocks[i] : 0, 1, 1};
      case COLL: {
        const int tx = tile_x(b->tile_variant), ty = tile_y(b->tile_variant);
        return {(int)cdiv(c->nx, tx), (int)cdiv(c->ny, ty), (int)cdiv(c->nz, b->zc)};
      }
      case INTERP: return {mem ? (int)cdiv(32ll * c->nn, NT) : 0, 1, 1};
      default: return {(int)(cdiv(c->N, NT) + cdiv(c->nn, NT)), 1, 1};
    }
  }

  // tile shape of a collide variant, read off the variant dispatch itself
  static int2 tile_of(int v) {
    int2 t = {32, 1};
    collide_variant<L>(v, [&](auto tx, auto ty, auto) {
      t = {decltype(tx)::value, decltype(ty)::value};
      return TLB_OK;
    });
    return t;
  }
  static int tile_x(int v) { return tile_of(v).x; }
  static int tile_y(int v) { return tile_of(v).y; }

  template <int MINB, class... Ops>
  static int occupancy_grid(int nt) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase<NT, MINB, BA, Ops...>, nt, 0);
    return std::max(1, per_sm);
  }

  // Virtual grids of every phase for the active instances; resident CTAs of
  // each phase kernel.
  tlb_status plan_phases(Batch* b) {
    const int n = (int)b->act.size();
    std::vector<int> h((size_t)Batch::NPH * Batch::MAXOPS * std::max(n, 1) * 4, 0);
    for (int ph = 0; ph < Batch::NPH; ++ph) {
      const std::vector<int> ops = phase_ops(ph);
      int start = 0;
      int* t = h.data() + (size_t)ph * Batch::MAXOPS * std::max(n, 1) * 4;
      for (size_t k = 0; k < ops.size(); ++k)
        for (int j = 0; j < n; ++j) {
          int3 g = op_grid(b, b->act[j], ops[k]);
          const long long cnt = (long long)g.x * g.y * g.z;
          if (cnt <= 0) g = {0, 1, 1};
          if ((long long)start + std::max(0ll, cnt) >= (1ll << 31)) {
            set_error("batch: more than 2^31 virtual blocks in one phase");
            return TLB_ERR_ARG;
          }
          int* e = t + 4 * (k * n + j);
          e[0] = g.x;
          e[1] = g.y;
          e[2] = g.z;
          e[3] = start;
          start += (int)std::max(0ll, cnt);
        }
      b->ph_ent[ph] = (int)ops.size() * n;
      b->ph_total[ph] = start;
    }
    TLB_CUDA(cudaMemcpyAsync(b->ptr<char>(b->vg), h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    TLB_CUDA(cudaStreamSynchronize(b->stream));
    int dev = 0, sms = 0;
    TLB_CUDA(cudaGetDevice(&dev));
    TLB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int ph = 0; ph < Batch::NPH; ++ph) {
      int per_sm = 1;
      switch (ph) {
        case 0: per_sm = occupancy_grid<8, OpPre<MODE>, OpMoments<L, MODE>, OpGeometry<MODE>, OpBrickCount<MODE>>(NT); break;
        case 1: per_sm = occupancy_grid<5, OpNodeForces<MODE>, OpScatter<MODE>, OpBrickCompact<MODE>>(NT); break;
        case 2: per_sm = occupancy_grid<8, OpBand<MODE>, OpBrickFill<MODE>>(NT); break;
        case 3: per_sm = occupancy_grid<8, OpSpread<MODE>, OpFill<MODE>>(NT); break;
        case 4: per_sm = collide_occupancy(b->tile_variant); break;
        case 5: per_sm = occupancy_grid<8, OpInterp<L, MODE>>(NT); break;
        default: per_sm = occupancy_grid<4, OpResidual<L, MODE>>(NT); break;
      }
      b->ph_grid[ph] = std::max(1, std::min(b->ph_total[ph], per_sm * sms));
    }
    return TLB_OK;
  }

  template <int TX, int TY, int FORM>
  static int collide_occ() {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm,
        k_phase<collide_block<FORM, TX, TY>(), collide_threads<FORM>() / collide_block<FORM, TX, TY>(), BA,
                OpCollide<L, MODE, TX, TY, FORM>>,
        collide_block<FORM, TX, TY>(), 0);
    return std::max(1, per_sm);
  }
  static int collide_occupancy(int v) {
    int per_sm = 1;
    collide_variant<L>(v, [&](auto tx, auto ty, auto fm) {
      per_sm = collide_occ<decltype(tx)::value, decltype(ty)::value, decltype(fm)::value>();
      return TLB_OK;
    });
    return per_sm;
  }


  template <int TX, int TY, int FORM>
  static tlb_status launch_collide_t(Batch* b, const BA* A, const int4* vg, cudaStream_t s) {
    const int n = (int)b->act.size();
    k_phase<collide_block<FORM, TX, TY>(), collide_threads<FORM>() / collide_block<FORM, TX, TY>(), BA,
            OpCollide<L, MODE, TX, TY, FORM>>
        <<<b->ph_grid[4], collide_block<FORM, TX, TY>(), 0, s>>>(A, vg, n, b->ph_ent[4], b->ph_total[4]);
    b->launches++;
    return cuda_check(cudaGetLastError(), "k_phase collide");
  }
  static tlb_status launch_collide(Batch* b, const BA* A, const int4* vg, cudaStream_t s) {
    return collide_variant<L>(b->tile_variant, [&](auto tx, auto ty, auto fm) {
      return launch_collide_t<decltype(tx)::value, decltype(ty)::value, decltype(fm)::value>(b, A, vg, s);
    });
  }

  const int4* vg_of(Batch* b, int ph) const {
    const int n = std::max(1, (int)b->act.size());
    return b->ptr<int4>(b->vg) + (size_t)ph * Batch::MAXOPS * n;
  }

  tlb_status launch_phase(Batch* b, int ph, const BA* A, cudaStream_t s) {
    if (b->ph_total[ph] == 0) return TLB_OK;
    const int n = (int)b->act.size();
    const int4* vg = vg_of(b, ph);
    const int g = b->ph_grid[ph], ne = b->ph_ent[ph], tot = b->ph_total[ph];
    switch (ph) {
      case 0:
        k_phase<NT, 8, BA, OpPre<MODE>, OpMoments<L, MODE>, OpGeometry<MODE>, OpBrickCount<MODE>>
            <<<g, NT, 0, s>>>(A, vg, n, ne, tot);
        break;
      case 1:
        k_phase<NT, 5, BA, OpNodeForces<MODE>, OpScatter<MODE>, OpBrickCompact<MODE>><<<g, NT, 0, s>>>(A, vg, n, ne, tot);
        break;
      case 2: k_phase<NT, 8, BA, OpBand<MODE>, OpBrickFill<MODE>><<<g, NT, 0, s>>>(A, vg, n, ne, tot); break;
      case 3: k_phase<NT, 8, BA, OpSpread<MODE>, OpFill<MODE>><<<g, NT, 0, s>>>(A, vg, n, ne, tot); break;
      case 4: return launch_collide(b, A, vg, s);
      case 5: k_phase<NT, 8, BA, OpInterp<L, MODE>><<<g, NT, 0, s>>>(A, vg, n, ne, tot); break;
      default: k_phase<NT, 4, BA, OpResidual<L, MODE>><<<g, NT, 0, s>>>(A, vg, n, ne, tot); break;
    }
    b->launches++;
    return cuda_check(cudaGetLastError(), "k_phase");
  }

  // One step of every active instance with the argument table of parity q.
  tlb_status launch_step(Batch* b, int q, cudaStream_t s) {
    const BA* A = b->ptr<BA>(b->targs[q]);
    for (int ph = 0; ph < 6; ++ph) {
      tlb_status st = launch_phase(b, ph, A, s);
      if (st != TLB_OK) return st;
    }
    return TLB_OK;
  }

  // Argument tables of the active instances: parity q reads the buffer
  // cur ^ q of each instance.
  tlb_status upload_tables(Batch* b) {
    const int n = (int)b->act.size();
    for (int q = 0; q < 2; ++q) {
      std::vector<BA> t((size_t)std::max(n, 1));
      for (int j = 0; j < n; ++j) {
        Ctx* c = b->inst[b->act[j]];
        BA& a = t[j];
        a.lb = I::lbargs(c, c->cur ^ q);
        a.lb.zc = b->zc;
        a.lb.jm = variant_t1(b->tile_variant) ? c->ptr<typename Prec<MODE>::Real>(c->L.jm) : nullptr;
        a.ib = I::ibargs(c);
        a.rp = I::resptrs(c, b->ptr<unsigned long long>(b->res) + 4 * (size_t)b->act[j]);
      }
      TLB_CUDA(cudaMemcpyAsync(b->ptr<char>(b->targs[q]), t.data(), (size_t)n * sizeof(BA), cudaMemcpyHostToDevice,
                               b->stream));
      TLB_CUDA(cudaStreamSynchronize(b->stream));
    }
    return TLB_OK;
  }

  // Markers overwritten since the last step: rebuild the box accumulator
  // from scratch (the snapshot is taken by the first phase of the step).
  tlb_status refresh_boxes(Batch* b) {
    for (int i : b->act) {
      Ctx* c = b->inst[i];
      if (!c->box_stale || c->nn == 0) continue;
      IBArgs<Real> a = I::ibargs(c);
      TLB_CUDA(cudaMemsetAsync(a.box, 0x7F, 6 * sizeof(int), b->stream));
      k_box<Real><<<cdiv(c->nn, 128), 128, 0, b->stream>>>(a);
      b->launches++;
      TLB_CUDA(cudaGetLastError());
      c->box_stale = false;
    }
    return TLB_OK;
  }

  tlb_status capture(Batch* b) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    long keep = b->launches;
    TLB_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    tlb_status st = launch_step(b, 0, b->cap);
    if (st == TLB_OK) st = launch_step(b, 1, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    b->graph_launches = b->launches - keep;
    b->launches = keep;
    if (st != TLB_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    TLB_CUDA(e);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    TLB_CUDA(e);
    b->graph_dirty = false;
    return TLB_OK;
  }

  tlb_status prepare(Batch* b) {
    if (b->graph_dirty) {
      tlb_status st = plan_phases(b);
      if (st != TLB_OK) return st;
    }
    tlb_status st = upload_tables(b);
    if (st != TLB_OK) return st;
    if (b->graph_dirty && !b->act.empty()) {
      st = capture(b);
      if (st != TLB_OK) return st;
    }
    return refresh_boxes(b);
  }

  tlb_status step(Batch* b, long n) override {
    if (b->act.empty() || n == 0) return TLB_OK;
    tlb_status st = prepare(b);
    if (st != TLB_OK) return st;
    // the graph's two steps leave every buffer parity as it was
    for (long k = 0; k + 1 < n; k += 2) {
      TLB_CUDA(cudaGraphLaunch(b->graph, b->stream));
      b->launches += b->graph_launches;
    }
    if (n & 1) {
      st = launch_step(b, 0, b->stream);
      if (st != TLB_OK) return st;
      for (int i : b->act) b->inst[i]->cur ^= 1;
    }
    for (int i : b->act) b->inst[i]->t += n;
    return TLB_OK;
  }

  tlb_status profile(Batch* b, long n, double* ms) override {
    for (int ph = 0; ph < 6; ++ph) ms[ph] = 0;
    if (b->act.empty() || n == 0) return TLB_OK;
    tlb_status st = prepare(b);
    if (st != TLB_OK) return st;
    cudaEvent_t ev[7];
    for (int k = 0; k < 7; ++k) TLB_CUDA(cudaEventCreate(&ev[k]));
    for (long k = 0; k < n && st == TLB_OK; ++k) {
      const BA* A = b->ptr<BA>(b->targs[k & 1]);
      for (int ph = 0; ph < 6 && st == TLB_OK; ++ph) {
        cudaEventRecord(ev[ph], b->stream);
        st = launch_phase(b, ph, A, b->stream);
      }
      cudaEventRecord(ev[6], b->stream);
      cudaEventSynchronize(ev[6]);
      for (int ph = 0; ph < 6; ++ph) {
        float t = 0;
        cudaEventElapsedTime(&t, ev[ph], ev[ph + 1]);
        ms[ph] += t;
      }
    }
    for (int k = 0; k < 7; ++k) cudaEventDestroy(ev[k]);
    if (st != TLB_OK) return st;
    if (n & 1)
      for (int i : b->act) b->inst[i]->cur ^= 1;
    for (int i : b->act) b->inst[i]->t += n;
    return TLB_OK;
  }

  tlb_status residual(Batch* b) override {
    if (b->act.empty()) return TLB_OK;
    tlb_status st = prepare(b);
    if (st != TLB_OK) return st;
    TLB_CUDA(cudaMemsetAsync(b->ptr<char>(b->res), 0, b->res.bytes, b->stream));
    return launch_phase(b, 6, b->ptr<BA>(b->targs[0]), b->stream);
  }

  // Collide tile shape and z chunk of the batch, timed on the current state
  // of the active instances (the collide reads one buffer and writes the
  // other, so repeats leave the state unchanged).
  tlb_status autotune(Batch* b, int* variant, int* zc) override {
    if (b->act.empty()) return TLB_OK;
    cudaEvent_t e0, e1;
    TLB_CUDA(cudaEventCreate(&e0));
    TLB_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bv = b->tile_variant, bz = b->zc;
    int nzmax = 0;
    for (int i : b->act) nzmax = std::max(nzmax, b->inst[i]->nz);
    const std::vector<int> zcs = z_chunk_candidates(nzmax);
    tlb_status st = TLB_OK;
    // the moments of the current state feed the collide (only the moments:
    // the first phase of a step would also consume the marker box)
    for (int i : b->act) {
      Ctx* c = b->inst[i];
      LBArgs<MODE> la = I::lbargs(c, c->cur);
      la.jm = c->ptr<typename Prec<MODE>::Real>(c->L.jm);
      k_moments<L, MODE><<<cdiv(c->N, 256), 256, 0, b->stream>>>(la);
      b->launches++;
      TLB_CUDA(cudaGetLastError());
    }
    auto all_ok = [&](int v) {
      for (int i : b->act)
        if (!b->inst[i]->variant_ok(v)) return false;
      return true;
    };
    for (int v = 0; v < COLLIDE_NVAR && st == TLB_OK; ++v)
      for (size_t zi = 0; zi < zcs.size() && st == TLB_OK; ++zi) {
        if (!all_ok(v)) continue;
        b->tile_variant = v;
        b->zc = zcs[zi];
        b->graph_dirty = true;
        st = plan_phases(b);
        if (st == TLB_OK) st = upload_tables(b);
        if (st == TLB_OK) st = launch_collide(b, b->ptr<BA>(b->targs[0]), vg_of(b, 4), b->stream);
        float tmin = 1e30f;
        for (int r = 0; r < 2 && st == TLB_OK; ++r) {
          cudaEventRecord(e0, b->stream);
          st = launch_collide(b, b->ptr<BA>(b->targs[0]), vg_of(b, 4), b->stream);
          cudaEventRecord(e1, b->stream);
          cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          tmin = std::min(tmin, ms);
        }
        if (st == TLB_OK && tmin < best) {
          best = tmin;
          bv = v;
          bz = zcs[zi];
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TLB_OK) return st;
    b->tile_variant = bv;
    b->zc = bz;
    b->graph_dirty = true;
    if (variant) *variant = bv;
    if (zc) *zc = bz;
    TLB_CUDA(cudaStreamSynchronize(b->stream));
    return TLB_OK;
  }
};
