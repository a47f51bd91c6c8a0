// Fifth-generation tensor core primitives (tcgen05, sm_100 family) in inline
// PTX: tensor memory (TMEM) allocation, the single-thread MMA with operands
// in shared memory, completion through an mbarrier, and the epilogue load of
// the fp32 accumulator from TMEM into registers.
//
// Operands are K-major without swizzle: a matrix is a grid of "core
// matrices" of 8 rows x 16 bytes (8 bf16 along K), each 128 contiguous bytes
// (row i at +16 i).  Its shared-memory descriptor holds the start address,
// the byte step between core matrices adjacent along K and the byte step
// between core matrices adjacent along M (or N), all in units of 16 bytes.
#pragma once
#include <stdint.h>

namespace umma {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, K step, M/N step (bytes,
// multiples of 16, below 256 KiB), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t desc(unsigned addr, unsigned kstep, unsigned mstep) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((kstep >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((mstep >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: bf16 A and B (both K-major), fp32
// accumulator, M x N.
template <int M, int N>
__device__ __forceinline__ constexpr unsigned idesc_bf16() {
  static_assert(M == 64 || M == 128, "M");
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "N");
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

// TMEM columns: a power of two, at least 32.
__host__ __device__ constexpr int tmem_cols(int n) {
  return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : (n <= 256 ? 256 : 512)));
}

// Warp-wide (all 32 lanes of one warp): allocate / free `ncols` TMEM
// columns; the base address is written to shared memory at `slot`.
__device__ __forceinline__ void tmem_alloc(unsigned* slot, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(unsigned taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// shared-memory writes of this thread (plain stores or cp.async) made
// visible to the tensor core's reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// D[tmem] (+)= A B^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(unsigned d_tmem, uint64_t a, uint64_t b, unsigned idesc, bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"((unsigned)accumulate)
      : "memory");
}

// The mbarrier at `bar` receives one arrival when every tcgen05 operation
// this thread issued before has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Wait until phase `parity` of the mbarrier has completed, at most `limit`
// polls; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long limit) {
  const unsigned a = smem_u32(bar);
  for (long it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive fp32 columns of the accumulator row held by this thread's
// TMEM lane (warp w of the CTA reads lanes 32 w .. 32 w + 31).
__device__ __forceinline__ void ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16-byte asynchronous copy global -> shared; zero fill when !valid
// (nothing is read then).
__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

}  // namespace umma

namespace umma {

// mbarrier arrival (count 1 of this thread), and arrival that also expects
// `tx` bytes of asynchronous copies to complete on it.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(tx) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// Non-blocking poll of phase `parity`, at most `limit` polls (with a short
// sleep between them after the first thousand); false if it gave up.
__device__ __forceinline__ bool mbar_poll(uint64_t* bar, unsigned parity, long limit) {
  const unsigned a = smem_u32(bar);
  for (long it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.test_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 1024) __nanosleep(64);
  }
  return false;
}

// Tiled TMA loads (global -> shared, completion counted in bytes on `bar`);
// the tensor map lives in kernel parameter space.  Out-of-volume elements
// of the box read as zero.
__device__ __forceinline__ void tma_load_5d(void* dst, const void* tmap, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace umma
