// Learned warm start: a 3D convolutional encoder-decoder that maps the plain
// initial state of a capsule-on-interface run and its parameters to a guess
// of the equilibrium (corrections of phi and psi and a displacement field
// sampled at the markers), trained by this file's own forward and backward
// kernels.  The lattice Boltzmann + immersed boundary relaxation then starts
// from that guess.  Not in the paper; see include/tlb.h for the network.
//
// Layout: activations channels-last bf16 [B][E_l^3][C] (C a multiple of 16);
// activation gradients fp32 of the same shape; master weights, gradients and
// Adam moments fp32 in the order W[tap][ci][co], b[co] per conv; the GEMMs
// read bf16 weight copies K-contiguous per output: Wf[co][tap*Ci + ci] for
// the forward pass and Wd[ci][tap*Co + co] (taps mirrored) for the data
// gradient.  Every convolution is an implicit GEMM on the tensor cores
// (mma.sync m16n8k16 bf16, fp32 accumulation).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tlb_ctx.h"
#include "tlb_umma.cuh"

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------ GEMM core
__device__ __forceinline__ void mma_bf16(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int TM = 64;    // GEMM rows per CTA (4 warps x 16)
constexpr int TK = 16;    // K per stage
constexpr int SK = 24;    // shared row stride (bf16), 48 bytes: 16-byte aligned, conflict-light
constexpr int YC = 16;    // output channels: dphi, dpsi, displacement (3), 11 unused

// One 16 x BN slab of a warp: A rows arow (k contiguous), B rows n (k contiguous).
template <int BN>
__device__ __forceinline__ void warp_mma(const bf16 (*As)[SK], const bf16 (*Bs)[SK], int arow, float (*acc)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  unsigned a[4];
  a[0] = *reinterpret_cast<const unsigned*>(&As[arow + g][2 * t]);
  a[1] = *reinterpret_cast<const unsigned*>(&As[arow + g + 8][2 * t]);
  a[2] = *reinterpret_cast<const unsigned*>(&As[arow + g][2 * t + 8]);
  a[3] = *reinterpret_cast<const unsigned*>(&As[arow + g + 8][2 * t + 8]);
#pragma unroll
  for (int j = 0; j < BN / 8; ++j) {
    unsigned b[2];
    b[0] = *reinterpret_cast<const unsigned*>(&Bs[j * 8 + g][2 * t]);
    b[1] = *reinterpret_cast<const unsigned*>(&Bs[j * 8 + g][2 * t + 8]);
    mma_bf16(acc[j], a, b);
  }
}

struct Vox {
  int b, z, y, x;
};
__device__ __forceinline__ Vox vox_of(long long v, int El) {
  Vox r;
  r.x = (int)(v % El);
  r.y = (int)((v / El) % El);
  r.z = (int)((v / ((long long)El * El)) % El);
  r.b = (int)(v / ((long long)El * El * El));
  return r;
}
// neighbour of voxel p at tap (27: offsets -1..1 per axis, z slowest; 1: itself), -1 outside
__device__ __forceinline__ long long nbr(const Vox& p, int tap, int taps, int El) {
  int dz = 0, dy = 0, dx = 0;
  if (taps == 27) {
    dz = tap / 9 - 1;
    dy = (tap / 3) % 3 - 1;
    dx = tap % 3 - 1;
  }
  const int z = p.z + dz, y = p.y + dy, x = p.x + dx;
  if (z < 0 || z >= El || y < 0 || y >= El || x < 0 || x >= El) return -1;
  return (((long long)p.b * El + z) * El + y) * El + x;
}

// out[v][co] = sum_{tap, ci} in[nbr(v, tap)][ci] W[tap][ci][co]  (+ bias),
// stored as bf16 relu(.) (RELU) or fp32.  in: [nvox][Ci] bf16; Wk: [Co][taps*Ci].
template <int BN, bool RELU>
__global__ void __launch_bounds__(128) k_conv(const bf16* __restrict__ in, int Ci, int El, long long nvox, int taps,
                                              const bf16* __restrict__ Wk, const float* __restrict__ bias, int Co,
                                              void* __restrict__ out) {
  __shared__ __align__(16) bf16 As[2][TM][SK];
  __shared__ __align__(16) bf16 Bs[2][BN][SK];
  const int tid = threadIdx.x, w = tid >> 5;
  const long long m0 = (long long)blockIdx.x * TM;
  const int n0 = blockIdx.y * BN;
  const int K = taps * Ci, nk = K / TK, cpt = Ci / TK;
  // A: thread -> (row, 8-channel half); B: thread -> (n, half) for tid < 2 BN
  const int ar = tid >> 1, ah = tid & 1;
  const long long av = m0 + ar;
  Vox p{0, 0, 0, 0};
  if (av < nvox) p = vox_of(av, El);
  uint4 ra, rb;
  auto load = [&](int kc) {
    const int tap = kc / cpt, ci0 = (kc % cpt) * TK + ah * 8;
    ra = make_uint4(0, 0, 0, 0);
    if (av < nvox) {
      const long long q = nbr(p, tap, taps, El);
      if (q >= 0) ra = *reinterpret_cast<const uint4*>(in + q * Ci + ci0);
    }
    if (tid < 2 * BN) rb = *reinterpret_cast<const uint4*>(Wk + (long long)(n0 + (tid >> 1)) * K + kc * TK + (tid & 1) * 8);
  };
  auto store = [&](int s) {
    *reinterpret_cast<uint4*>(&As[s][ar][ah * 8]) = ra;
    if (tid < 2 * BN) *reinterpret_cast<uint4*>(&Bs[s][tid >> 1][(tid & 1) * 8]) = rb;
  };
  float acc[BN / 8][4];
#pragma unroll
  for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  load(0);
  store(0);
  __syncthreads();
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc & 1;
    if (kc + 1 < nk) load(kc + 1);
    warp_mma<BN>(As[s], Bs[s], w * 16, acc);
    if (kc + 1 < nk) store(s ^ 1);
    __syncthreads();
  }
  const int lane = tid & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const long long v = m0 + w * 16 + g + half * 8;
    if (v >= nvox) continue;
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) {
      const int n = n0 + j * 8 + 2 * t;
      float o0 = acc[j][half * 2], o1 = acc[j][half * 2 + 1];
      if (bias) {
        o0 += bias[n];
        o1 += bias[n + 1];
      }
      if (RELU) {
        __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(o0, 0.f), fmaxf(o1, 0.f));
        *reinterpret_cast<__nv_bfloat162*>(static_cast<bf16*>(out) + v * Co + n) = h;
      } else {
        *reinterpret_cast<float2*>(static_cast<float*>(out) + v * Co + n) = make_float2(o0, o1);
      }
    }
  }
}

// 3x3x3 convolution on bricks: a CTA computes an 8x4x4 brick of output
// voxels (128 GEMM rows, 4 warps x 2 m16 tiles) for BN output channels.  Per
// chunk of 16 input channels it stages the brick's input with a halo of 1
// (10x6x6 voxels, zero outside the volume) and the chunk's weights of all 27
// taps in shared memory once, then runs the 27 taps as shifted views of the
// staged input.  Rows are 48 bytes apart, so the fragment loads of 8
// consecutive rows hit distinct banks.
constexpr int BRX = 8, BRY = 4, BRZ = 4, HX = BRX + 2, HY = BRY + 2, HZ = BRZ + 2, HV = HX * HY * HZ;

template <int BN>
constexpr int conv3_smem() { return (HV + 27 * BN) * SK * 2; }

template <int BN, bool RELU>
__global__ void __launch_bounds__(128) k_conv3(const bf16* __restrict__ in, int Ci, int El, int nbatch,
                                               const bf16* __restrict__ Wk, const float* __restrict__ bias, int Co,
                                               void* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  bf16 (*Xs)[SK] = reinterpret_cast<bf16 (*)[SK]>(smem);
  bf16 (*Ws)[SK] = reinterpret_cast<bf16 (*)[SK]>(smem + HV * SK * 2);
  const int bpx = (El + BRX - 1) / BRX, bpy = (El + BRY - 1) / BRY, bpz = (El + BRZ - 1) / BRZ;
  int bid = blockIdx.x;
  const int bx = bid % bpx;
  bid /= bpx;
  const int by = bid % bpy;
  bid /= bpy;
  const int bz = bid % bpz;
  const int b = bid / bpz;
  if (b >= nbatch) return;
  const int x0 = bx * BRX, y0 = by * BRY, z0 = bz * BRZ, n0 = blockIdx.y * BN;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int K = 27 * Ci;
  float acc[2][BN / 8][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) acc[mt][j][0] = acc[mt][j][1] = acc[mt][j][2] = acc[mt][j][3] = 0.f;
  // input-tile voxel of GEMM row r at tap offset (0..2 per axis)
  auto tile_vox = [](int r, int dz, int dy, int dx) {
    return ((r / (BRX * BRY) + dz) * HY + (r / BRX) % BRY + dy) * HX + r % BRX + dx;
  };
  for (int ci0 = 0; ci0 < Ci; ci0 += 16) {
    for (int i = tid; i < HV * 2; i += 128) {
      const int v = i >> 1, h = i & 1;
      const int X = x0 - 1 + v % HX, Y = y0 - 1 + (v / HX) % HY, Z = z0 - 1 + v / (HX * HY);
      uint4 val = make_uint4(0, 0, 0, 0);
      if (X >= 0 && X < El && Y >= 0 && Y < El && Z >= 0 && Z < El)
        val = *reinterpret_cast<const uint4*>(in + ((((long long)b * El + Z) * El + Y) * El + X) * Ci + ci0 + h * 8);
      *reinterpret_cast<uint4*>(&Xs[v][h * 8]) = val;
    }
    for (int i = tid; i < 27 * BN * 2; i += 128) {
      const int row = i >> 1, h = i & 1, tap = row / BN, n = row % BN;
      *reinterpret_cast<uint4*>(&Ws[row][h * 8]) =
          *reinterpret_cast<const uint4*>(Wk + (long long)(n0 + n) * K + tap * Ci + ci0 + h * 8);
    }
    __syncthreads();
#pragma unroll 1
    for (int tap = 0; tap < 27; ++tap) {
      const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
      unsigned a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r0 = (w * 2 + mt) * 16 + g;
        const int v0 = tile_vox(r0, dz, dy, dx), v1 = tile_vox(r0 + 8, dz, dy, dx);
        a[mt][0] = *reinterpret_cast<const unsigned*>(&Xs[v0][2 * t]);
        a[mt][1] = *reinterpret_cast<const unsigned*>(&Xs[v1][2 * t]);
        a[mt][2] = *reinterpret_cast<const unsigned*>(&Xs[v0][2 * t + 8]);
        a[mt][3] = *reinterpret_cast<const unsigned*>(&Xs[v1][2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < BN / 8; ++j) {
        unsigned bb[2];
        bb[0] = *reinterpret_cast<const unsigned*>(&Ws[tap * BN + j * 8 + g][2 * t]);
        bb[1] = *reinterpret_cast<const unsigned*>(&Ws[tap * BN + j * 8 + g][2 * t + 8]);
        mma_bf16(acc[0][j], a[0], bb);
        mma_bf16(acc[1][j], a[1], bb);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int r = (w * 2 + mt) * 16 + g + half * 8;
      const int X = x0 + r % BRX, Y = y0 + (r / BRX) % BRY, Z = z0 + r / (BRX * BRY);
      if (X >= El || Y >= El || Z >= El) continue;
      const long long v = (((long long)b * El + Z) * El + Y) * El + X;
#pragma unroll
      for (int j = 0; j < BN / 8; ++j) {
        const int n = n0 + j * 8 + 2 * t;
        float o0 = acc[mt][j][half * 2], o1 = acc[mt][j][half * 2 + 1];
        if (bias) {
          o0 += bias[n];
          o1 += bias[n + 1];
        }
        if (RELU) {
          __nv_bfloat162 hv = __floats2bfloat162_rn(fmaxf(o0, 0.f), fmaxf(o1, 0.f));
          *reinterpret_cast<__nv_bfloat162*>(static_cast<bf16*>(out) + v * Co + n) = hv;
        } else {
          *reinterpret_cast<float2*>(static_cast<float*>(out) + v * Co + n) = make_float2(o0, o1);
        }
      }
    }
}

// 3x3x3 convolution on the fifth-generation tensor cores (tcgen05): a CTA
// computes ZB planes of 8 (x) x 16 (y) output voxels, one M = 128 GEMM tile
// per plane (row r: x = r % 8, y = r / 8), for BN output channels, the ZB
// accumulators side by side in tensor memory.  Per chunk of 16 input
// channels the input brick with its halo of 1 (10 x 18 x (ZB + 2) voxels,
// zero outside the volume) and the chunk's weights of all 27 taps are copied
// into shared memory (cp.async, two stages: the next chunk's copy runs under
// this chunk's products), laid out as K-major core matrices:
//   input   A[kh][voxel][8 channels]  (voxel = (z HY + y) HX + x),
//   weights B[kh][tap BN + n][8 channels].
// A tap's operand is then a strided view of the staged brick: its 16 row
// groups of 8 voxels (one y row each) lie HX voxels apart, so one
// descriptor per tap and plane serves, and one thread issues 27 ZB products
// of 128 x BN x 16 per chunk.  The epilogue reads each warp's 32 rows back
// from tensor memory, adds the bias, applies relu and stores channels-last.
// Waits on the tensor core give up after a bounded number of polls (status
// bit 1 then) and the tensor memory is freed on every path.
constexpr int TC_HX = 10, TC_HY = 18;
template <int BN, int ZB>
constexpr int tc_stage_bytes() { return 2 * TC_HX * TC_HY * (ZB + 2) * 16 + 2 * 27 * BN * 16; }
template <int BN, int ZB>
constexpr int tc_smem() { return 2 * tc_stage_bytes<BN, ZB>() + 32; }

// The 27 ZB products of one chunk of 16 input channels, issued by one
// thread, tap by tap: plane zp and tap (dz, dy, dx) read the staged brick from voxel
// ((zp + dz) HY + dy) HX + dx on.  A descriptor's start-address field is its
// low 14 bits (16-byte units, below 2^14 for any shared address), so each
// product's descriptors are the chunk's base descriptors plus constants.
template <int BN, int ZB, int HX, int HY, int HV>
__device__ __forceinline__ void conv3_products(unsigned As, unsigned Bs, unsigned dtmem, bool acc0) {
  constexpr unsigned IDESC = umma::idesc_bf16<128, BN>();
  const uint64_t a0 = umma::desc(As, HV * 16, HX * 16), b0 = umma::desc(Bs, 27 * BN * 16, 128);
  // consecutive products go to different planes' accumulators, so that
  // they do not wait on one another
#pragma unroll
  for (int tap = 0; tap < 27; ++tap) {
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const uint64_t at = a0 + (uint64_t)((dz * HY + dy) * HX + dx), bt = b0 + (uint64_t)(tap * BN);
#pragma unroll
    for (int zp = 0; zp < ZB; ++zp)
      umma::mma_bf16(dtmem + zp * BN, at + (uint64_t)(zp * HY * HX), bt, IDESC, acc0 || tap > 0);
  }
}

template <int BN, int ZB, bool RELU>
__global__ void __launch_bounds__(128) k_conv3_tc(const bf16* __restrict__ in, int Ci, int El, int nbatch,
                                                  const bf16* __restrict__ Wk, const float* __restrict__ bias,
                                                  int Co, void* __restrict__ out, unsigned* __restrict__ status) {
  constexpr int HX = TC_HX, HY = TC_HY, HZ = ZB + 2, HV = HX * HY * HZ;
  constexpr int ABYTES = 2 * HV * 16, STAGE = tc_stage_bytes<BN, ZB>();
  constexpr int NCOL = umma::tmem_cols(ZB * BN);
  constexpr long POLL = 1L << 22;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE);
  unsigned* tslot = reinterpret_cast<unsigned*>(smem + 2 * STAGE + 16);
  const int bpx = (El + 7) / 8, bpy = (El + 15) / 16, bpz = (El + ZB - 1) / ZB;
  int bid = blockIdx.x;
  const int bx = bid % bpx;
  bid /= bpx;
  const int by = bid % bpy;
  bid /= bpy;
  const int bz = bid % bpz;
  const int b = bid / bpz;
  if (b >= nbatch) return;
  const int x0 = bx * 8, y0 = by * 16, z0 = bz * ZB, n0 = blockIdx.y * BN;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int K = 27 * Ci, nck = Ci / 16;

  if (w == 0) umma::tmem_alloc(tslot, NCOL);
  if (tid == 0) {
    umma::mbar_init(&bar[0], 1);
    umma::mbar_init(&bar[1], 1);
  }
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const unsigned tmem = *tslot;

  auto stage = [&](int s, int ck) {
    unsigned char* As = smem + s * STAGE;
    unsigned char* Bs = As + ABYTES;
    const int ci0 = ck * 16;
    for (int i = tid; i < 2 * HV; i += 128) {
      const int v = i >> 1, kh = i & 1;
      const int X = x0 - 1 + v % HX, Y = y0 - 1 + (v / HX) % HY, Z = z0 - 1 + v / (HX * HY);
      const bool ok = X >= 0 && X < El && Y >= 0 && Y < El && Z >= 0 && Z < El;
      const bf16* src = ok ? in + ((((long long)b * El + Z) * El + Y) * El + X) * Ci + ci0 + kh * 8 : in;
      umma::cp16(As + (kh * HV + v) * 16, src, ok);
    }
    for (int i = tid; i < 2 * 27 * BN; i += 128) {
      const int row = i >> 1, kh = i & 1, tap = row / BN, n = row % BN;
      umma::cp16(Bs + (kh * 27 * BN + row) * 16, Wk + (long long)(n0 + n) * K + tap * Ci + ci0 + kh * 8, true);
    }
  };

  bool ok = true;
  stage(0, 0);
  umma::cp_commit();
  for (int ck = 0; ck < nck; ++ck) {
    const int s = ck & 1;
    if (ck + 1 < nck) {
      // the other stage was read by the products of chunk ck - 1
      if (ck >= 1 && ok) ok = umma::mbar_wait(&bar[s ^ 1], ((ck - 1) >> 1) & 1, POLL);
      stage(s ^ 1, ck + 1);
      umma::cp_commit();
      umma::cp_wait<1>();
    } else {
      umma::cp_wait<0>();
    }
    umma::fence_proxy_async();
    __syncthreads();
    if (tid == 0 && ok) {
      umma::fence_after_sync();
      const unsigned As = umma::smem_u32(smem + s * STAGE), Bs = As + ABYTES;
      conv3_products<BN, ZB, HX, HY, HV>(As, Bs, tmem, ck > 0);
      umma::commit(&bar[s]);
    }
  }
  if (ok) ok = umma::mbar_wait(&bar[(nck - 1) & 1], ((nck - 1) >> 1) & 1, POLL);
  if (!ok) atomicOr(status, 1u);
  umma::fence_after_sync();
  if (__all_sync(0xffffffffu, ok)) {
    const int r = 32 * w + lane, X = x0 + r % 8, Y = y0 + r / 8;
    for (int zp = 0; zp < ZB; ++zp) {
      const int Z = z0 + zp;
      const bool in_vol = X < El && Y < El && Z < El;
      const long long v = (((long long)b * El + Z) * El + Y) * El + X;
#pragma unroll 1
      for (int j0 = 0; j0 < BN; j0 += 16) {
        float o[16];
        umma::ld16(tmem + ((unsigned)(32 * w) << 16) + zp * BN + j0, o);
        if (!in_vol) continue;
        const int n = n0 + j0;
        if (bias)
#pragma unroll
          for (int i = 0; i < 16; ++i) o[i] += bias[n + i];
        if (RELU) {
          uint4 pk[2];
          unsigned* u = reinterpret_cast<unsigned*>(pk);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(o[2 * i], 0.f), fmaxf(o[2 * i + 1], 0.f));
            u[i] = *reinterpret_cast<unsigned*>(&h);
          }
          uint4* dst = reinterpret_cast<uint4*>(static_cast<bf16*>(out) + v * Co + n);
          dst[0] = pk[0];
          dst[1] = pk[1];
        } else {
          float4* dst = reinterpret_cast<float4*>(static_cast<float*>(out) + v * Co + n);
#pragma unroll
          for (int i = 0; i < 4; ++i) dst[i] = make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
        }
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (w == 0) umma::tmem_free(tmem, NCOL);
}

// The same 3x3x3 convolution as a persistent, warp-specialised tcgen05
// pipeline fed by the tensor memory accelerator (TMA):
//  - warp 4 (one thread) loads each chunk of 16 input channels of a work
//    item (a brick of ZB planes of 8 x 16 output voxels and BN output
//    channels) with four tiled TMA copies: the input brick with its halo as
//    two 5D boxes of 8 channels x 10 x 18 x (ZB + 2) voxels (zero outside
//    the volume) and the weights as two 3D boxes of 8 channels x BN outputs
//    x 27 taps, landing in exactly the K-major core-matrix layouts of
//    k_conv3_tc, into one of S shared-memory stages;
//  - warp 5 (one thread) issues the 27 ZB products of each chunk into one of
//    two tensor-memory accumulators and frees the stage through an mbarrier
//    when they complete;
//  - warps 0..3 drain the other accumulator (bias, relu, channels-last
//    store) while the next item accumulates.
// Every wait is bounded (status bit 1 when one gave up; the roles then stop
// and the tensor memory is freed).
constexpr int TMA_THREADS = 192;
// stages: as many as fit in 227 KiB of shared memory, 2 to 4
template <int BN, int ZB>
constexpr int tma_stages() {
  return (232448 - 1280) / tc_stage_bytes<BN, ZB>() >= 4 ? 4 : ((232448 - 1280) / tc_stage_bytes<BN, ZB>() >= 3 ? 3 : 2);
}
template <int BN, int ZB>
constexpr int tma_smem() { return 1024 + tma_stages<BN, ZB>() * tc_stage_bytes<BN, ZB>() + 256; }

template <int BN, int ZB, bool RELU>
__global__ void __launch_bounds__(TMA_THREADS) k_conv3_tma(const __grid_constant__ CUtensorMap tin,
                                                           const __grid_constant__ CUtensorMap tw, int Ci, int El,
                                                           int nbatch, const float* __restrict__ bias, int Co,
                                                           void* __restrict__ out, unsigned* __restrict__ status) {
  constexpr int HX = TC_HX, HY = TC_HY, HZ = ZB + 2, HV = HX * HY * HZ;
  constexpr int ABYTES = 2 * HV * 16, STAGE = tc_stage_bytes<BN, ZB>(), S = tma_stages<BN, ZB>();
  constexpr int NCOL = umma::tmem_cols(2 * ZB * BN);
  constexpr long POLL = 1L << 24;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024 - (umma::smem_u32(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * STAGE);
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  unsigned* tslot = reinterpret_cast<unsigned*>(acc_empty + 2);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int bpx = (El + 7) / 8, bpy = (El + 15) / 16, bpz = (El + ZB - 1) / ZB;
  const int nbr = bpx * bpy * bpz * nbatch, ntile = Co / BN, items = nbr * ntile, nck = Ci / 16;

  if (w == 5) umma::tmem_alloc(tslot, NCOL);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      umma::mbar_init(&acc_full[a], 1);
      umma::mbar_init(&acc_empty[a], 128);
    }
    umma::mbar_init_fence();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const unsigned tmem = *tslot;
  auto item_coords = [&](int it, int& x0, int& y0, int& z0, int& b, int& n0) {
    const int t = it % ntile;
    int r = it / ntile;
    x0 = (r % bpx) * 8;
    r /= bpx;
    y0 = (r % bpy) * 16;
    r /= bpy;
    z0 = (r % bpz) * ZB;
    b = r / bpz;
    n0 = t * BN;
  };
  bool ok = true;
  if (w == 4) {
    if (lane == 0) {  // producer
      long g = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int x0, y0, z0, b, n0;
        item_coords(it, x0, y0, z0, b, n0);
        for (int ck = 0; ck < nck && ok; ++ck, ++g) {
          const int s = (int)(g % S);
          if (g >= S) ok = umma::mbar_poll(&empty[s], (unsigned)((g / S - 1) & 1), POLL);
          if (!ok) break;
          unsigned char* As = smem + s * STAGE;
          unsigned char* Bs = As + ABYTES;
          umma::mbar_expect_tx(&full[s], (unsigned)STAGE);
          for (int kh = 0; kh < 2; ++kh) {
            umma::tma_load_5d(As + kh * HV * 16, &tin, ck * 16 + kh * 8, x0 - 1, y0 - 1, z0 - 1, b, &full[s]);
            umma::tma_load_3d(Bs + kh * 27 * BN * 16, &tw, ck * 16 + kh * 8, n0, 0, &full[s]);
          }
        }
      }
    }
  } else if (w == 5) {
    if (lane == 0) {  // tensor-core issue
      long g = 0;
      int j = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x, ++j) {
        const int acc = j & 1;
        if (j >= 2) ok = umma::mbar_poll(&acc_empty[acc], (unsigned)((j / 2 - 1) & 1), POLL);
        if (!ok) break;
        umma::fence_after_sync();
        const unsigned dbase = tmem + acc * ZB * BN;
        for (int ck = 0; ck < nck && ok; ++ck, ++g) {
          const int s = (int)(g % S);
          ok = umma::mbar_poll(&full[s], (unsigned)((g / S) & 1), POLL);
          if (!ok) break;
          umma::fence_after_sync();
          const unsigned As = umma::smem_u32(smem + s * STAGE), Bs = As + ABYTES;
          conv3_products<BN, ZB, HX, HY, HV>(As, Bs, dbase, ck > 0);
          umma::commit(&empty[s]);
        }
        if (ok) umma::commit(&acc_full[acc]);
      }
    }
  } else {  // epilogue: warp w holds accumulator rows 32 w .. 32 w + 31
    int j = 0;
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x, ++j) {
      const int acc = j & 1;
      ok = umma::mbar_poll(&acc_full[acc], (unsigned)((j / 2) & 1), POLL);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      umma::fence_after_sync();
      int x0, y0, z0, b, n0;
      item_coords(it, x0, y0, z0, b, n0);
      const int r = 32 * w + lane, X = x0 + r % 8, Y = y0 + r / 8;
      for (int zp = 0; zp < ZB; ++zp) {
        const int Z = z0 + zp;
        const bool in_vol = X < El && Y < El && Z < El;
        const long long v = (((long long)b * El + Z) * El + Y) * El + X;
#pragma unroll 1
        for (int j0 = 0; j0 < BN; j0 += 16) {
          float o[16];
          umma::ld16(tmem + ((unsigned)(32 * w) << 16) + acc * ZB * BN + zp * BN + j0, o);
          if (!in_vol) continue;
          const int n = n0 + j0;
          if (bias)
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] += bias[n + i];
          if (RELU) {
            uint4 pk[2];
            unsigned* u = reinterpret_cast<unsigned*>(pk);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(o[2 * i], 0.f), fmaxf(o[2 * i + 1], 0.f));
              u[i] = *reinterpret_cast<unsigned*>(&h);
            }
            uint4* dst = reinterpret_cast<uint4*>(static_cast<bf16*>(out) + v * Co + n);
            dst[0] = pk[0];
            dst[1] = pk[1];
          } else {
            float4* dst = reinterpret_cast<float4*>(static_cast<float*>(out) + v * Co + n);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
          }
        }
      }
      umma::fence_before_sync();
      umma::mbar_arrive(&acc_empty[acc]);
    }
  }
  if (!ok) atomicOr(status, 1u);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (w == 5) umma::tmem_free(tmem, NCOL);
}

// Shared-memory 8x8 b16 matrices, transposed on load (ldmatrix .trans): lane
// l gives the row address of matrix l / 8; each row holds 8 consecutive b16.
__device__ __forceinline__ void ldsm_x4_t(unsigned* r, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned* r, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

// Weight gradient of a 3x3x3 conv on bricks: dW[tap][ci][co] = sum over
// voxels v of in[v + offset(tap)][ci] gz[v][co], a GEMM with rows (ci), columns
// (co) and the voxels as K.  A CTA owns 16 input channels (blockIdx.z), BN
// output channels (blockIdx.y) and the bricks blockIdx.x, blockIdx.x +
// gridDim.x, ...; per brick it stages the input with its halo and gz in
// shared memory and warp w accumulates the taps w, w + 4, ... over the
// brick's 128 voxels.  Operands are read transposed from the channels-last
// rows with ldmatrix.  Writes part[blockIdx.x][tap][ci][co] (fixed order of
// bricks per CTA, so the sums are deterministic).
template <int BN>
constexpr int gs_stride() { return BN + 8; }
template <int BN>
constexpr int wgrad3_smem() { return HV * SK * 2 + 128 * gs_stride<BN>() * 2; }

template <int BN>
__global__ void __launch_bounds__(128) k_wgrad3(const bf16* __restrict__ in, int Ci, int El, int nbatch,
                                                const bf16* __restrict__ gz, int Co, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int GS = gs_stride<BN>();
  bf16 (*Xs)[SK] = reinterpret_cast<bf16 (*)[SK]>(smem);
  bf16 (*Gs)[GS] = reinterpret_cast<bf16 (*)[GS]>(smem + HV * SK * 2);
  const int bpx = (El + BRX - 1) / BRX, bpy = (El + BRY - 1) / BRY, bpz = (El + BRZ - 1) / BRZ;
  const int nbr = bpx * bpy * bpz * nbatch;
  const int n0 = blockIdx.y * BN, ci0 = blockIdx.z * 16;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  constexpr int NTW = 7;  // taps per warp: w, w + 4, ... below 27
  float acc[NTW][BN / 8][4];
#pragma unroll
  for (int s = 0; s < NTW; ++s)
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) acc[s][j][0] = acc[s][j][1] = acc[s][j][2] = acc[s][j][3] = 0.f;
  // ldmatrix row of this lane: voxel kk of a 16-voxel k-step, column half
  const int lrow = (lane & 7) + ((lane >> 4) << 3), lcol = ((lane >> 3) & 1) * 8;
  for (int bb = blockIdx.x; bb < nbr; bb += gridDim.x) {
    int bid = bb;
    const int bx = bid % bpx;
    bid /= bpx;
    const int by = bid % bpy;
    bid /= bpy;
    const int bz = bid % bpz;
    const int b = bid / bpz;
    const int x0 = bx * BRX, y0 = by * BRY, z0 = bz * BRZ;
    for (int i = tid; i < HV * 2; i += 128) {
      const int v = i >> 1, h = i & 1;
      const int X = x0 - 1 + v % HX, Y = y0 - 1 + (v / HX) % HY, Z = z0 - 1 + v / (HX * HY);
      uint4 val = make_uint4(0, 0, 0, 0);
      if (X >= 0 && X < El && Y >= 0 && Y < El && Z >= 0 && Z < El)
        val = *reinterpret_cast<const uint4*>(in + ((((long long)b * El + Z) * El + Y) * El + X) * Ci + ci0 + h * 8);
      *reinterpret_cast<uint4*>(&Xs[v][h * 8]) = val;
    }
    for (int i = tid; i < 128 * (BN / 8); i += 128) {
      const int r = i / (BN / 8), q = i % (BN / 8);
      const int X = x0 + r % BRX, Y = y0 + (r / BRX) % BRY, Z = z0 + r / (BRX * BRY);
      uint4 val = make_uint4(0, 0, 0, 0);
      if (X < El && Y < El && Z < El)
        val = *reinterpret_cast<const uint4*>(gz + ((((long long)b * El + Z) * El + Y) * El + X) * Co + n0 + q * 8);
      *reinterpret_cast<uint4*>(&Gs[r][q * 8]) = val;
    }
    __syncthreads();
#pragma unroll 1
    for (int k0 = 0; k0 < 128; k0 += 16) {
      unsigned bf[BN / 8][2];
#pragma unroll
      for (int j = 0; j < BN / 8; ++j) ldsm_x2_t(bf[j], &Gs[k0 + (lane & 15)][j * 8]);
      const int kk = k0 + lrow;
      const int lz = kk / (BRX * BRY), ly = (kk / BRX) % BRY, lx = kk % BRX;
#pragma unroll
      for (int s = 0; s < NTW; ++s) {
        const int tap = w + 4 * s;
        if (tap < 27) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          unsigned af[4];
          ldsm_x4_t(af, &Xs[((lz + dz) * HY + ly + dy) * HX + lx + dx][lcol]);
#pragma unroll
          for (int j = 0; j < BN / 8; ++j) mma_bf16(acc[s][j], af, bf[j]);
        }
      }
    }
    __syncthreads();
  }
  float* P = part + (size_t)blockIdx.x * 27 * Ci * Co;
#pragma unroll
  for (int s = 0; s < NTW; ++s) {
    const int tap = w + 4 * s;
    if (tap >= 27) continue;
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) {
      const int n = n0 + j * 8 + 2 * t;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int ci = ci0 + g + half * 8;
        float* dst = P + ((size_t)tap * Ci + ci) * Co + n;
        dst[0] = acc[s][j][half * 2];
        dst[1] = acc[s][j][half * 2 + 1];
      }
    }
  }
}

// out[i] = sum over k < nsplit of part[k * n + i] (i < n), in two passes
// whose grouping is fixed (so the result does not depend on timing): pass 1
// (k_sum_groups) adds the splits of each group of SPLIT_GROUP into the
// group's first row, in place; pass 2 (k_sum_splits with step SPLIT_GROUP)
// adds the groups' rows.  Each thread keeps eight running sums (split k to
// sum k mod 8) combined in a fixed tree, so eight loads are in flight.
constexpr int SPLIT_GROUP = 16;
__device__ __forceinline__ float sum_rows(const float* __restrict__ part, int k0, int k1, int step, long long n,
                                          long long i) {
  float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int k = k0;
  for (; k + 8 * step <= k1; k += 8 * step)
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] += part[(size_t)(k + j * step) * n + i];
  for (int j = 0; k < k1; k += step, ++j) a[j & 7] += part[(size_t)k * n + i];
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}
__global__ void k_sum_groups(float* __restrict__ part, int nsplit, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k0 = blockIdx.y * SPLIT_GROUP;
  if (i >= n || k0 >= nsplit) return;
  part[(size_t)k0 * n + i] = sum_rows(part, k0, min(nsplit, k0 + SPLIT_GROUP), 1, n, i);
}
__global__ void k_sum_splits(const float* __restrict__ part, int nsplit, long long n, int step, float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = sum_rows(part, 0, nsplit, step, n, i);
}

// Column sums of gz (the bias gradient): block b sums voxels [b chunk,
// (b + 1) chunk); thread (tx, ty) of its TX x TY threads (TX = min(Co, 256))
// takes channels tx, tx + TX, .. of voxels ty, ty + TY, ..; the TY partial
// sums of a channel are then added in ty order (fixed, so deterministic).
__global__ void __launch_bounds__(256) k_colsum(const bf16* __restrict__ gz, long long V, int Co, long long chunk,
                                                float* __restrict__ part) {
  __shared__ float sm[256];
  const int TX = Co < 256 ? Co : 256, TY = 256 / TX;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const long long v0 = (long long)blockIdx.x * chunk, v1 = min(V, v0 + chunk);
  for (int c0 = 0; c0 < Co; c0 += TX) {
    float s = 0.f;
    const bool live = ty < TY && c0 + tx < Co;
    if (live)
      for (long long v = v0 + ty; v < v1; v += TY) s += __bfloat162float(gz[v * Co + c0 + tx]);
    __syncthreads();
    sm[threadIdx.x] = s;
    __syncthreads();
    if (ty == 0 && c0 + tx < Co) {
      float t = 0.f;
      for (int k = 0; k < TY; ++k) t += sm[k * TX + tx];
      part[(size_t)blockIdx.x * Co + c0 + tx] = t;
    }
  }
}

// Weight (and bias) gradient of one conv, split over voxel ranges:
//   part[split][m][n] = sum_{v in range} A[m][v] gz[v][n]
// with rows m = tap*Ci + ci: A[m][v] = in[nbr(v, tap)][ci], and one extra row
// m = taps*Ci of ones (its sums are the bias gradient).
template <int BN>
__global__ void __launch_bounds__(128) k_wgrad(const bf16* __restrict__ in, int Ci, int El, long long nvox, int taps,
                                               const bf16* __restrict__ gz, int Co, long long vchunk,
                                               float* __restrict__ part) {
  __shared__ __align__(16) bf16 As[2][TM][SK];
  __shared__ __align__(16) bf16 Bs[2][BN][SK];
  const int tid = threadIdx.x, w = tid >> 5;
  const int M = taps * Ci + 1;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * BN;
  const long long v0 = (long long)blockIdx.z * vchunk;
  const long long v1 = min(nvox, v0 + vchunk);
  const int nk = (int)((v1 - v0 + TK - 1) / TK);
  // A: thread -> (voxel k = tid / 8, rows gq*8 .. +7); B: thread -> (voxel, 8 columns)
  const int ak = tid >> 3, aq = tid & 7;
  const int am = m0 + aq * 8;
  const int atap = am / Ci, aci = am % Ci;
  const int bcols = BN / 8, bk = tid / bcols, bq = tid % bcols;
  uint4 ra, rb;
  auto load = [&](int kc) {
    const long long v = v0 + (long long)kc * TK + ak;
    ra = make_uint4(0, 0, 0, 0);
    if (v < v1) {
      if (am + 8 <= M - 1) {
        const long long q = nbr(vox_of(v, El), atap, taps, El);
        if (q >= 0) ra = *reinterpret_cast<const uint4*>(in + q * Ci + aci);
      } else if (am <= M - 1) {  // the block of 8 rows holding the ones row
        __align__(16) bf16 one[8];
        for (int j = 0; j < 8; ++j) one[j] = __float2bfloat16_rn(am + j == M - 1 ? 1.f : 0.f);
        ra = *reinterpret_cast<const uint4*>(one);
      }
    }
    rb = make_uint4(0, 0, 0, 0);
    const long long vb = v0 + (long long)kc * TK + bk;
    if (tid < TK * bcols && vb < v1) rb = *reinterpret_cast<const uint4*>(gz + vb * Co + n0 + bq * 8);
  };
  auto store = [&](int s) {
    const bf16* e = reinterpret_cast<const bf16*>(&ra);
#pragma unroll
    for (int j = 0; j < 8; ++j) As[s][aq * 8 + j][ak] = e[j];
    if (tid < TK * bcols) {
      const bf16* f = reinterpret_cast<const bf16*>(&rb);
#pragma unroll
      for (int j = 0; j < 8; ++j) Bs[s][bq * 8 + j][bk] = f[j];
    }
  };
  float acc[BN / 8][4];
#pragma unroll
  for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  if (nk > 0) {
    load(0);
    store(0);
  }
  __syncthreads();
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc & 1;
    if (kc + 1 < nk) load(kc + 1);
    warp_mma<BN>(As[s], Bs[s], w * 16, acc);
    if (kc + 1 < nk) store(s ^ 1);
    __syncthreads();
  }
  const int lane = tid & 31, g = lane >> 2, t = lane & 3;
  float* P = part + (size_t)blockIdx.z * M * Co;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int m = m0 + w * 16 + g + half * 8;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) {
      const int n = n0 + j * 8 + 2 * t;
      P[(size_t)m * Co + n] = acc[j][half * 2];
      P[(size_t)m * Co + n + 1] = acc[j][half * 2 + 1];
    }
  }
}

// dW (rows < M-1) and db (row M-1) from the split partials, summed in split order.
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nsplit, int M, int Co, float* __restrict__ dW,
                               float* __restrict__ db) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)M * Co) return;
  float s = 0.f;
  for (int k = 0; k < nsplit; ++k) s += part[(size_t)k * M * Co + i];
  const int m = (int)(i / Co);
  if (m < M - 1) dW[i] = s;
  else db[i - (long long)(M - 1) * Co] = s;
}

// ------------------------------------------------------------ elementwise
// 2x2x2 average pooling, [B][El^3][C] -> [B][(El/2)^3][C], bf16.
// voxel index -> (b, z, y, x) on an El^3 grid, 32-bit (fewer than 2^31 voxels)
struct Vox32 {
  unsigned b, z, y, x;
};
__device__ __forceinline__ Vox32 vox32(unsigned v, unsigned E) {
  Vox32 r;
  r.x = v % E;
  v /= E;
  r.y = v % E;
  v /= E;
  r.z = v % E;
  r.b = v / E;
  return r;
}

// 2x2x2 average pool, eight channels per thread (C is a multiple of 16).
__global__ void k_pool_fwd(const bf16* __restrict__ in, int El, int C, long long nout, bf16* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int G = C >> 3;
  if (i >= nout * G) return;
  const int g = (int)(i % G);
  const unsigned v = (unsigned)(i / G), E = (unsigned)El;
  const Vox32 p = vox32(v, E / 2);
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int d = 0; d < 8; ++d) {
    const unsigned q = ((p.b * E + 2 * p.z + (d >> 2)) * E + 2 * p.y + ((d >> 1) & 1)) * E + 2 * p.x + (d & 1);
    const uint4 w = *reinterpret_cast<const uint4*>(in + (long long)q * C + 8 * g);
    const bf16* h = reinterpret_cast<const bf16*>(&w);
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(h[k]);
  }
  uint4 o;
  unsigned* u = reinterpret_cast<unsigned*>(&o);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat162 b2 = __floats2bfloat162_rn(s[2 * k] * 0.125f, s[2 * k + 1] * 0.125f);
    u[k] = *reinterpret_cast<unsigned*>(&b2);
  }
  *reinterpret_cast<uint4*>(out + (long long)v * C + 8 * g) = o;
}

// g_in[child] += g_out[parent] / 8 (fp32).
__global__ void k_pool_bwd(const float* __restrict__ gout, int El, int C, long long nin, float* __restrict__ gin) {
  // four channels per thread (C is a multiple of 16)
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int G = C >> 2;
  if (i >= nin * G) return;
  const int g = (int)(i % G);
  const unsigned v = (unsigned)(i / G), E = (unsigned)El, Eh = E / 2;
  const Vox32 p = vox32(v, E);
  const unsigned q = ((p.b * Eh + p.z / 2) * Eh + p.y / 2) * Eh + p.x / 2;
  const float4 a = *reinterpret_cast<const float4*>(gout + (long long)q * C + 4 * g);
  float4* dst = reinterpret_cast<float4*>(gin + (long long)v * C + 4 * g);
  float4 b = *dst;
  b.x += 0.125f * a.x;
  b.y += 0.125f * a.y;
  b.z += 0.125f * a.z;
  b.w += 0.125f * a.w;
  *dst = b;
}

// cat[v] = [up2(d)[v] (C1) | e[v] (C2)], bf16.
__global__ void k_cat_fwd(const bf16* __restrict__ d, int C1, const bf16* __restrict__ e, int C2, int El, long long n,
                          bf16* __restrict__ cat) {
  // one thread per voxel and group of 8 channels (16 bytes; C1, C2 are
  // multiples of 16); 32-bit voxel arithmetic (n < 2^31 voxels)
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int G = (C1 + C2) >> 3;
  if (i >= n * G) return;
  const int g = (int)(i % G);
  const unsigned v = (unsigned)(i / G);
  uint4 val;
  if (8 * g >= C1) {
    val = *reinterpret_cast<const uint4*>(e + (long long)v * C2 + (8 * g - C1));
  } else {
    const unsigned E = (unsigned)El, Eh = E / 2;
    const unsigned x = v % E, r = v / E, y = r % E, r2 = r / E, z = r2 % E, b = r2 / E;
    const unsigned q = ((b * Eh + z / 2) * Eh + y / 2) * Eh + x / 2;
    val = *reinterpret_cast<const uint4*>(d + (long long)q * C1 + 8 * g);
  }
  *reinterpret_cast<uint4*>(cat + (long long)v * (C1 + C2) + 8 * g) = val;
}

// From g_cat: g_e += skip part (per fine voxel); g_d += sum over the 8 children (per coarse voxel).
__global__ void k_cat_bwd_skip(const float* __restrict__ gcat, int C1, int C2, long long n, float* __restrict__ ge) {
  // four channels per thread (C1, C2 are multiples of 16)
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int G = C2 >> 2;
  if (i >= n * G) return;
  const int g = (int)(i % G);
  const long long v = i / G;
  const float4 a = *reinterpret_cast<const float4*>(gcat + v * (C1 + C2) + C1 + 4 * g);
  float4* dst = reinterpret_cast<float4*>(ge + v * C2 + 4 * g);
  float4 b = *dst;
  b.x += a.x;
  b.y += a.y;
  b.z += a.z;
  b.w += a.w;
  *dst = b;
}
__global__ void k_cat_bwd_up(const float* __restrict__ gcat, int C1, int C2, int El, long long ncoarse,
                             float* __restrict__ gd) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int G = C1 >> 2;
  if (i >= ncoarse * G) return;
  const int g = (int)(i % G);
  const unsigned v = (unsigned)(i / G), E = (unsigned)El;
  const Vox32 p = vox32(v, E / 2);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int d = 0; d < 8; ++d) {
    const unsigned q = ((p.b * E + 2 * p.z + (d >> 2)) * E + 2 * p.y + ((d >> 1) & 1)) * E + 2 * p.x + (d & 1);
    const float4 a = *reinterpret_cast<const float4*>(gcat + (long long)q * (C1 + C2) + 4 * g);
    s.x += a.x;
    s.y += a.y;
    s.z += a.z;
    s.w += a.w;
  }
  float4* dst = reinterpret_cast<float4*>(gd + (long long)v * C1 + 4 * g);
  float4 b = *dst;
  b.x += s.x;
  b.y += s.y;
  b.z += s.z;
  b.w += s.w;
  *dst = b;
}

// gz = g * relu'(h) as bf16 (h > 0 where the stored activation is positive).
// gz = bf16(h > 0 ? g : 0) (or bf16(g)), eight elements per thread (n is a
// multiple of 16: channels come in multiples of 16).
__global__ void k_relu_bwd(const float* __restrict__ g, const bf16* __restrict__ h, long long n, bf16* __restrict__ gz) {
  const long long i = 8 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  const float4 g0 = *reinterpret_cast<const float4*>(g + i), g1 = *reinterpret_cast<const float4*>(g + i + 4);
  const uint4 hv = *reinterpret_cast<const uint4*>(h + i);
  const bf16* hb = reinterpret_cast<const bf16*>(&hv);
  const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
  uint4 o;
  unsigned* u = reinterpret_cast<unsigned*>(&o);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat162 p = __floats2bfloat162_rn(__bfloat162float(hb[2 * k]) > 0.f ? gv[2 * k] : 0.f,
                                              __bfloat162float(hb[2 * k + 1]) > 0.f ? gv[2 * k + 1] : 0.f);
    u[k] = *reinterpret_cast<unsigned*>(&p);
  }
  *reinterpret_cast<uint4*>(gz + i) = o;
}

__global__ void k_to_bf16(const float* __restrict__ g, long long n, bf16* __restrict__ o) {
  const long long i = 8 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  const float4 g0 = *reinterpret_cast<const float4*>(g + i), g1 = *reinterpret_cast<const float4*>(g + i + 4);
  uint4 r;
  unsigned* u = reinterpret_cast<unsigned*>(&r);
  const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat162 p = __floats2bfloat162_rn(gv[2 * k], gv[2 * k + 1]);
    u[k] = *reinterpret_cast<unsigned*>(&p);
  }
  *reinterpret_cast<uint4*>(o + i) = r;
}

// Field loss: gy[v][0..1] = 2/(B V) (y - target), gy[v][2..15] = 0, and the
// marker loss's fixed-point accumulators of v cleared (gfix, if not NULL);
// per-block FP64 partial sums of the squared errors.
__global__ void k_loss_fields(const float* __restrict__ y, const float* __restrict__ tphi, const float* __restrict__ tpsi,
                              long long n, double scale, float* __restrict__ gy, long long* __restrict__ gfix,
                              double* __restrict__ part) {
  __shared__ double sm[256];
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0;
  if (v < n) {
    const float d0 = y[v * YC] - tphi[v], d1 = y[v * YC + 1] - tpsi[v];
    e = (double)d0 * d0 + (double)d1 * d1;
    gy[v * YC] = (float)(2.0 * scale * d0);
    gy[v * YC + 1] = (float)(2.0 * scale * d1);
    for (int c = 2; c < YC; ++c) gy[v * YC + c] = 0.f;
    if (gfix)
      for (int a = 0; a < 3; ++a) gfix[3 * v + a] = 0;
  }
  sm[threadIdx.x] = e;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// Trilinear sampling of channels 2..4 of y at X (clamped to [0, E-1]); the
// 8 corner weights and indices of one point.
struct Tri {
  long long idx[8];
  float w[8];
};
__device__ __forceinline__ Tri tri_of(float x, float y, float z, int E) {
  Tri T;
  x = fminf(fmaxf(x, 0.f), E - 1.f);
  y = fminf(fmaxf(y, 0.f), E - 1.f);
  z = fminf(fmaxf(z, 0.f), E - 1.f);
  const int ix = min((int)floorf(x), E - 2), iy = min((int)floorf(y), E - 2), iz = min((int)floorf(z), E - 2);
  const float fx = x - ix, fy = y - iy, fz = z - iz;
  for (int d = 0; d < 8; ++d) {
    const int dx = d & 1, dy = (d >> 1) & 1, dz = d >> 2;
    T.w[d] = (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy) * (dz ? fz : 1.f - fz);
    T.idx[d] = ((long long)(iz + dz) * E + (iy + dy)) * E + (ix + dx);
  }
  return T;
}

// The marker loss's gradient is scattered in fixed point (steps of
// 2^-GFIX_BITS) with integer atomics: the sums do not depend on the order of
// the additions, so a training step is reproducible bit for bit.  Each
// contribution is clamped to +-2^GFIX_CLAMP, far above any gradient of this
// loss (2 lambda / (3 markers) times an offset error), so that the few
// hundred contributions a voxel can receive stay inside the 2^(63 -
// GFIX_BITS) range.
constexpr int GFIX_BITS = 48, GFIX_CLAMP = 8;

// Marker loss of sample b: offsets = trilinear(y2..4)(X0); the gradient is
// added, scattered with the trilinear weights, into the fixed-point
// accumulators gfix[v][0..2] of the sample; FP64 partial sums of the loss.
__global__ void k_loss_nodes(const float* __restrict__ y, const float* __restrict__ X0, const float* __restrict__ toff,
                             int nn, int E, double scale, long long* __restrict__ gfix, double* __restrict__ part) {
  __shared__ double sm[256];
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0;
  if (l < nn) {
    const Tri T = tri_of(X0[3 * l], X0[3 * l + 1], X0[3 * l + 2], E);
    for (int a = 0; a < 3; ++a) {
      float o = 0.f;
      for (int d = 0; d < 8; ++d) o += T.w[d] * y[T.idx[d] * YC + 2 + a];
      const float r = o - toff[3 * l + a];
      e += (double)r * r;
      const float gr = (float)(2.0 * scale * r);
      for (int d = 0; d < 8; ++d) {
        const double c = fmin(fmax((double)(gr * T.w[d]), -(double)(1 << GFIX_CLAMP)), (double)(1 << GFIX_CLAMP));
        const long long q = __double2ll_rn(c * (double)(1ll << GFIX_BITS));
        atomicAdd(reinterpret_cast<unsigned long long*>(gfix + 3 * T.idx[d] + a), (unsigned long long)q);
      }
    }
  }
  sm[threadIdx.x] = e;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// gy[v][2..4] = gfix[v][0..2] 2^-GFIX_BITS (the marker loss's gradient).
__global__ void k_loss_fold(const long long* __restrict__ gfix, long long n, float* __restrict__ gy) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double s = 1.0 / (double)(1ll << GFIX_BITS);
  for (int a = 0; a < 3; ++a) gy[v * YC + 2 + a] = (float)((double)gfix[3 * v + a] * s);
}

// Adam (Kingma and Ba 2015) on fp32 parameters; c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bf16 GEMM copies of one conv's weights W[tap][ci][co]:
// Wf[co][tap*Ci + ci] and Wd[ci][tap*Co + co] with the tap mirrored.
__global__ void k_weights(const float* __restrict__ W, int taps, int Ci, int Co, bf16* __restrict__ Wf,
                          bf16* __restrict__ Wd) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)taps * Ci * Co) return;
  const int co = (int)(i % Co), ci = (int)((i / Co) % Ci), tap = (int)(i / ((long long)Co * Ci));
  const bf16 w = __float2bfloat16_rn(W[i]);
  Wf[(long long)co * taps * Ci + (long long)tap * Ci + ci] = w;
  Wd[(long long)ci * taps * Co + (long long)(taps - 1 - tap) * Co + co] = w;
}

// Network input of one sample from a context's fields: phi0, psi0, the
// broadcast features, zeros.
__global__ void k_make_input(const float* __restrict__ phi, const float* __restrict__ psi, long long V, float f0,
                             float f1, float f2, float f3, float f4, bf16* __restrict__ x) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  __align__(16) bf16 c[16];
  const float fv[7] = {phi[v], psi[v], f0, f1, f2, f3, f4};
  for (int k = 0; k < 16; ++k) c[k] = __float2bfloat16_rn(k < 7 ? fv[k] : 0.f);
  reinterpret_cast<uint4*>(x + v * 16)[0] = reinterpret_cast<uint4*>(c)[0];
  reinterpret_cast<uint4*>(x + v * 16)[1] = reinterpret_cast<uint4*>(c)[1];
}

// ---- warm start of a context (see tlb_net_warm_start)
// Displacement of every marker: D_l = trilinear(y2..4)(X0_l) into D [nn][3],
// with FP64 partial sums of D for the mean translation.
__global__ void k_ws_disp(const double* __restrict__ X, int nn, const float* __restrict__ y, int E, float* __restrict__ D,
                          double* __restrict__ part) {
  __shared__ double sm[3][128];
  const int l = blockIdx.x * 128 + threadIdx.x;
  double a[3] = {0, 0, 0};
  if (l < nn) {
    const Tri T = tri_of((float)X[3 * l], (float)X[3 * l + 1], (float)X[3 * l + 2], E);
    for (int q = 0; q < 3; ++q) {
      float o = 0.f;
      for (int d = 0; d < 8; ++d) o += T.w[d] * y[T.idx[d] * YC + 2 + q];
      D[3 * l + q] = o;
      a[q] = o;
    }
  }
  for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[q * gridDim.x + blockIdx.x] = sm[q][0];
}

// X_l += T + ((D_l - T) . n_l) n_l: the mean translation T = tot / nn and the
// normal part of the rest, n_l the unit vertex pseudo-normal.
__global__ void k_ws_move(double* __restrict__ X, int nn, const float* __restrict__ D, const float* __restrict__ vn,
                          const double* __restrict__ tot) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nn) return;
  double T[3], n[3], r = 0, len = 0;
  for (int q = 0; q < 3; ++q) {
    T[q] = tot[q] / nn;
    n[q] = vn[3 * l + q];
    len += n[q] * n[q];
  }
  len = sqrt(len);
  for (int q = 0; q < 3; ++q) {
    n[q] = len > 0 ? n[q] / len : 0.0;
    r += ((double)D[3 * l + q] - T[q]) * n[q];
  }
  for (int q = 0; q < 3; ++q) X[3 * l + q] += T[q] + r * n[q];
}

// FP64 partial sums of the marker positions (their centroid).
__global__ void k_ws_centroid(const double* __restrict__ X, int nn, double* __restrict__ part) {
  __shared__ double sm[3][128];
  const int l = blockIdx.x * 128 + threadIdx.x;
  for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] = l < nn ? X[3 * l + q] : 0.0;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[q * gridDim.x + blockIdx.x] = sm[q][0];
}

// Volume projection of the moved membrane: X_l = c + s (X_l - c) about the
// centroid c = tot / nn with s = (V0 / V1)^(1/3), so that the capsule
// encloses the plain start's volume V0 again (the fluid inside is conserved
// by the method, so the prediction's shape change must not change it).
__global__ void k_ws_scale(double* __restrict__ X, int nn, const double* __restrict__ tot,
                           const double* __restrict__ v0, const double* __restrict__ v1) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nn) return;
  const double s = cbrt(v0[1] / v1[1]);
  for (int q = 0; q < 3; ++q) {
    const double c = tot[q] / nn;
    X[3 * l + q] = c + s * (X[3 * l + q] - c);
  }
}

__global__ void k_capsule_measures(const double* X, const int* E, const int* ecap, int ne, int NV, int ncap,
                                   double* out);

// Plain-start phase indicator of the C1/C2 fluid: s0 = phi0 / (1 - psi0)
// (the plain start has phi0 = (1 - psi0)(2 s - 1)), 0 where 1 - psi0 < 1e-6.
__device__ __forceinline__ double s0_of(float phi0, float psi0) {
  const double w = 1.0 - (double)psi0;
  return w > 1e-6 ? (double)phi0 / w : 0.0;
}

// The warm start restores the plain totals of psi and phi (the method
// conserves both) by moving interfaces, not by shifting bulk values: the
// corrections are weighted by 4 I (1 - I) (nonzero only across the
// membrane's profile) and by (1 - s^2)_+ (only across the C1/C2 interface),
// so that the bulk fluids start at their equilibrium compositions.
__device__ __forceinline__ double ws_wpsi(float I) { return 4.0 * (double)I * (1.0 - (double)I); }
__device__ __forceinline__ double ws_wphi(double s) { return fmax(0.0, 1.0 - s * s); }

// Block partial sums of nq values per cell, written to part[q][block].
template <int NQ, class F>
__device__ __forceinline__ void ws_block_sums(long long V, double* __restrict__ part, F cell) {
  __shared__ double sm[NQ][256];
  double a[NQ];
  for (int q = 0; q < NQ; ++q) a[q] = 0;
  for (long long v = (long long)blockIdx.x * 256 + threadIdx.x; v < V; v += (long long)gridDim.x * 256) cell(v, a);
  for (int q = 0; q < NQ; ++q) sm[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < NQ; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < NQ; ++q) part[q * gridDim.x + blockIdx.x] = sm[q][0];
}

// Pass 1: sums of phi0, psi0, I and 4 I (1 - I).
__global__ void k_ws_sums1(const float* __restrict__ phi, const float* __restrict__ psi, const float* __restrict__ I,
                           long long V, double* __restrict__ part) {
  ws_block_sums<4>(V, part, [&](long long v, double* a) {
    a[0] += phi[v];
    a[1] += psi[v];
    a[2] += I[v];
    a[3] += ws_wpsi(I[v]);
  });
}

__device__ __forceinline__ double ws_lpsi(const double* tot) {
  return tot[3] > 1e-12 ? (tot[1] - tot[2]) / tot[3] : 0.0;
}

// Pass 2, with psi = I + lpsi 4 I (1 - I) and s = s0 + y0: sums of
// (1 - psi) s and (1 - psi) (1 - s^2)_+.
__global__ void k_ws_sums2(const float* __restrict__ phi, const float* __restrict__ psi, const float* __restrict__ I,
                           const float* __restrict__ y, long long V, const double* __restrict__ tot,
                           double* __restrict__ part) {
  const double lpsi = ws_lpsi(tot);
  ws_block_sums<2>(V, part, [&](long long v, double* a) {
    const double w = 1.0 - ((double)I[v] + lpsi * ws_wpsi(I[v]));
    const double sv = s0_of(phi[v], psi[v]) + y[v * YC];
    a[0] += w * sv;
    a[1] += w * ws_wphi(sv);
  });
}

// Fields of the warm start: rho = 1 (the array holds rho - 1), psi = I +
// lpsi 4 I (1 - I), phi = (1 - psi)(s + lphi (1 - s^2)_+) with s = s0 + y0
// and lphi = (sum phi0 - tot2[0]) / tot2[1].
__global__ void k_ws_fields(float* __restrict__ rho, float* __restrict__ phi, float* __restrict__ psi,
                            const float* __restrict__ I, const float* __restrict__ y, long long V,
                            const double* __restrict__ tot, const double* __restrict__ tot2) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const double lpsi = ws_lpsi(tot);
  const double lphi = tot2[1] > 1e-12 ? (tot[0] - tot2[0]) / tot2[1] : 0.0;
  const double ps = (double)I[v] + lpsi * ws_wpsi(I[v]);
  const double sv = s0_of(phi[v], psi[v]) + y[v * YC];
  rho[v] = 0.f;
  phi[v] = (float)((1.0 - ps) * (sv + lphi * ws_wphi(sv)));
  psi[v] = (float)ps;
}

__global__ void k_sum_parts(const double* __restrict__ part, int nb, int nq, double* __restrict__ out) {
  __shared__ double sm[256];
  for (int q = 0; q < nq; ++q) {
    double a = 0;
    for (int i = threadIdx.x; i < nb; i += 256) a += part[q * nb + i];
    sm[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sm[0];
    __syncthreads();
  }
}

// ------------------------------------------------------------ host side
namespace {

struct Conv {
  int taps, ci, co, level;
  size_t w, b;       // offsets in the parameter vector
  size_t wf, wd;     // offsets (elements) in the bf16 weight copies
};

// A tensor of the network: channels-last, level l, C channels.
struct Ten {
  int level, C;
  size_t act;   // bf16 activation (elements offset), or SIZE_MAX
  size_t grad;  // fp32 gradient (elements offset), or SIZE_MAX
};

struct Net {
  tlb_net_desc d;
  cudaStream_t stream = nullptr;
  char* base = nullptr;
  size_t bytes = 0;
  std::vector<Conv> convs;
  size_t nparam = 0;
  // arena regions (byte offsets)
  size_t o_theta, o_grad, o_m, o_v, o_wf, o_wd, o_act, o_grad_act, o_gz, o_y, o_gy, o_part, o_gfix, o_lpart, o_misc;
  size_t n_wbf = 0, n_act = 0, n_gact = 0, n_gz = 0, n_part = 0;
  // tensors: x, per encoder level (a, e, pool input p), per decoder level (cat, b, d)
  Ten x, enc_a[4], enc_e[4], enc_p[4], dec_cat[4], dec_b[4], dec_d[4];
  long adam_t = 0;
  long launches = 0;
  int tc = 2;      // 3x3x3 convolutions: 0 mma.sync, 1 tcgen05 (cp.async staging), 2 tcgen05 fed by TMA
  int nsm = 1;     // streaming multiprocessors (persistent grids)
  unsigned* status() const { return reinterpret_cast<unsigned*>(base + o_misc + 64 * 8); }

  template <class T> T* at(size_t off) const { return reinterpret_cast<T*>(base + off); }
  long long vox(int level, int B) const {
    const long long El = d.edge >> level;
    return (long long)B * El * El * El;
  }
  int chan(int l) const { return d.base_channels << l; }
};

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

tlb_status check_desc(const tlb_net_desc* d) {
  if (!d) { set_error("net desc is NULL"); return TLB_ERR_ARG; }
  if (d->levels < 2 || d->levels > 4) { set_error("net: levels must be 2..4"); return TLB_ERR_ARG; }
  if (d->base_channels < 16 || d->base_channels % 16 || d->base_channels > 64) {
    set_error("net: base_channels must be 16, 32, 48 or 64");
    return TLB_ERR_ARG;
  }
  const int div = 1 << (d->levels - 1);
  if (d->edge < 2 * div || d->edge % div || d->edge > 256) {
    set_error("net: edge must be a multiple of 2^(levels-1), at least 2^levels and at most 256");
    return TLB_ERR_ARG;
  }
  if (d->max_batch < 1 || d->max_batch > 64) { set_error("net: max_batch must be 1..64"); return TLB_ERR_ARG; }
  if (d->max_nodes < 0 || d->max_nodes > (1 << 20)) { set_error("net: max_nodes must be 0..2^20"); return TLB_ERR_ARG; }
  return TLB_OK;
}

// Layers, parameter offsets, tensors and arena plan (offsets only).
void plan(Net& n) {
  const tlb_net_desc& d = n.d;
  const int L = d.levels, B = d.max_batch;
  n.convs.clear();
  size_t p = 0, wb = 0;
  auto conv = [&](int taps, int ci, int co, int level) {
    Conv c{taps, ci, co, level, p, p + (size_t)taps * ci * co, wb, 0};
    p += (size_t)taps * ci * co + co;
    wb += (size_t)taps * ci * co;
    n.convs.push_back(c);
  };
  conv(27, 16, n.chan(0), 0);
  conv(27, n.chan(0), n.chan(0), 0);
  for (int l = 1; l < L; ++l) {
    conv(27, n.chan(l - 1), n.chan(l), l);
    conv(27, n.chan(l), n.chan(l), l);
  }
  for (int l = L - 2; l >= 0; --l) {
    conv(27, n.chan(l + 1) + n.chan(l), n.chan(l), l);
    conv(27, n.chan(l), n.chan(l), l);
  }
  conv(1, n.chan(0), YC, 0);
  n.nparam = p;
  n.n_wbf = wb;
  for (Conv& c : n.convs) c.wd = c.wf;  // the two copies share offsets in their own arrays
  // activations (bf16) and activation gradients (fp32)
  size_t act = 0, gact = 0;
  auto ten = [&](int level, int C, bool want_grad) {
    Ten t{level, C, act, want_grad ? gact : (size_t)-1};
    act += (size_t)n.vox(level, B) * C;
    if (want_grad) gact += (size_t)n.vox(level, B) * C;
    return t;
  };
  n.x = ten(0, 16, false);
  for (int l = 0; l < L; ++l) {
    if (l > 0) n.enc_p[l] = ten(l, n.chan(l - 1), true);
    n.enc_a[l] = ten(l, n.chan(l), true);
    n.enc_e[l] = ten(l, n.chan(l), true);
  }
  for (int l = L - 2; l >= 0; --l) {
    n.dec_cat[l] = ten(l, n.chan(l + 1) + n.chan(l), true);
    n.dec_b[l] = ten(l, n.chan(l), true);
    n.dec_d[l] = ten(l, n.chan(l), true);
  }
  n.n_act = act;
  n.n_gact = gact;
  size_t gz = 0;
  for (const Conv& c : n.convs) gz = std::max(gz, (size_t)n.vox(c.level, B) * std::max(c.co, c.ci));
  n.n_gz = gz;
  // split-K partials of the weight gradient: at most 512 splits
  size_t part = 0;
  for (const Conv& c : n.convs) part = std::max(part, (size_t)(c.taps * c.ci + 1) * c.co);
  n.n_part = part * 512;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = al256(off + std::max<size_t>(bytes, 1));
    return o;
  };
  n.o_theta = take(n.nparam * 4);
  n.o_grad = take(n.nparam * 4);
  n.o_m = take(n.nparam * 4);
  n.o_v = take(n.nparam * 4);
  n.o_wf = take(n.n_wbf * 2);
  n.o_wd = take(n.n_wbf * 2);
  n.o_act = take(n.n_act * 2);
  n.o_grad_act = take(n.n_gact * 4);
  n.o_gz = take(n.n_gz * 2);
  n.o_y = take((size_t)n.vox(0, B) * YC * 4);
  n.o_gy = take((size_t)n.vox(0, B) * YC * 4);
  n.o_part = take(n.n_part * 4);
  n.o_gfix = take(d.max_nodes > 0 ? (size_t)n.vox(0, B) * 3 * 8 : 0);
  n.o_lpart = take((size_t)(nb(n.vox(0, B), 256) + (size_t)B * nb(d.max_nodes, 256) + 1024) * 8);
  n.o_misc = take(72 * 8);  // FP64 sums; the status word at double 64
  n.bytes = off;
}

// GEMM columns per CTA: the largest of 64, 32, 16 dividing the channel
// count (every channel count is a multiple of 16).
int tile_n(int C) { return C % 64 == 0 ? 64 : (C % 32 == 0 ? 32 : 16); }

#define NET_LAUNCHED(net, what)                                  \
  do {                                                           \
    (net)->launches++;                                           \
    tlb_status _s = cuda_check(cudaGetLastError(), what);        \
    if (_s != TLB_OK) return _s;                                 \
  } while (0)

template <int BN, bool RELU>
tlb_status launch_conv3_t(Net* n, const bf16* in, int Ci, int El, int B, const bf16* Wk, const float* bias, int Co,
                          void* out) {
  const long long bricks = (long long)((El + BRX - 1) / BRX) * ((El + BRY - 1) / BRY) * ((El + BRZ - 1) / BRZ) * B;
  constexpr int sm = conv3_smem<BN>();
  TLB_CUDA(cudaFuncSetAttribute(k_conv3<BN, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  k_conv3<BN, RELU><<<dim3((unsigned)bricks, Co / BN), 128, sm, n->stream>>>(in, Ci, El, B, Wk, bias, Co, out);
  NET_LAUNCHED(n, "k_conv3");
  return TLB_OK;
}

template <int BN, int ZB, bool RELU>
tlb_status launch_conv3_tc_t(Net* n, const bf16* in, int Ci, int El, int B, const bf16* Wk, const float* bias, int Co,
                             void* out) {
  const long long bricks = (long long)((El + 7) / 8) * ((El + 15) / 16) * ((El + ZB - 1) / ZB) * B;
  constexpr int sm = tc_smem<BN, ZB>();
  TLB_CUDA(cudaFuncSetAttribute(k_conv3_tc<BN, ZB, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  k_conv3_tc<BN, ZB, RELU><<<dim3((unsigned)bricks, Co / BN), 128, sm, n->stream>>>(in, Ci, El, B, Wk, bias, Co, out,
                                                                                     n->status());
  NET_LAUNCHED(n, "k_conv3_tc");
  return TLB_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    cudaGetLastError();
  }
  return fn;
}

// Tensor maps of a 3x3x3 convolution: the input [B][El^3][Ci] bf16 as 5D
// (channel, x, y, z, sample) with a box of 8 channels x 10 x 18 x (ZB + 2)
// voxels, the weights [Co][27 Ci] bf16 as 3D (channel, output, tap) with a
// box of 8 channels x BN outputs x 27 taps.
static tlb_status conv3_maps(const bf16* in, int Ci, int El, int B, int ZB, const bf16* Wk, int Co, int BN,
                             CUtensorMap* tin, CUtensorMap* tw) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) { set_error("net: cuTensorMapEncodeTiled is not available"); return TLB_ERR_CUDA; }
  const cuuint64_t e = (cuuint64_t)El, ci2 = (cuuint64_t)Ci * 2;
  const cuuint64_t gdim[5] = {(cuuint64_t)Ci, e, e, e, (cuuint64_t)B};
  const cuuint64_t gstr[4] = {ci2, ci2 * e, ci2 * e * e, ci2 * e * e * e};
  const cuuint32_t box[5] = {8, (cuuint32_t)TC_HX, (cuuint32_t)TC_HY, (cuuint32_t)(ZB + 2), 1};
  const cuuint32_t one[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(tin, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)in, gdim, gstr, box, one,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_error("net: input tensor map (" + std::to_string((int)r) + ")"); return TLB_ERR_CUDA; }
  const cuuint64_t wdim[3] = {(cuuint64_t)Ci, (cuuint64_t)Co, 27};
  const cuuint64_t wstr[2] = {27 * ci2, ci2};
  const cuuint32_t wbox[3] = {8, (cuuint32_t)BN, 27};
  r = enc(tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)Wk, wdim, wstr, wbox, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_error("net: weight tensor map (" + std::to_string((int)r) + ")"); return TLB_ERR_CUDA; }
  return TLB_OK;
}

template <int BN, int ZB, bool RELU>
tlb_status launch_conv3_tma_t(Net* n, const bf16* in, int Ci, int El, int B, const bf16* Wk, const float* bias,
                              int Co, void* out) {
  CUtensorMap tin, tw;
  if (tlb_status st = conv3_maps(in, Ci, El, B, ZB, Wk, Co, BN, &tin, &tw); st != TLB_OK) return st;
  const long long items = (long long)((El + 7) / 8) * ((El + 15) / 16) * ((El + ZB - 1) / ZB) * B * (Co / BN);
  constexpr int sm = tma_smem<BN, ZB>();
  TLB_CUDA(cudaFuncSetAttribute(k_conv3_tma<BN, ZB, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  const unsigned grid = (unsigned)std::min<long long>(items, n->nsm);
  k_conv3_tma<BN, ZB, RELU><<<grid, TMA_THREADS, sm, n->stream>>>(tin, tw, Ci, El, B, bias, Co, out, n->status());
  NET_LAUNCHED(n, "k_conv3_tma");
  return TLB_OK;
}

template <bool RELU>
tlb_status launch_conv(Net* n, const bf16* in, int Ci, int El, long long nvox, int taps, const bf16* Wk,
                       const float* bias, int Co, void* out) {
  if (taps == 27 && n->tc == 2) {  // TMA-fed persistent pipeline; columns per tile: 64, 32 or 16
    const int B = (int)(nvox / ((long long)El * El * El));
    // (8 planes, i.e. 8 independent accumulators per item, where the
    // tensor memory holds two sets of them)
    if (Co % 64 == 0) return launch_conv3_tma_t<64, 4, RELU>(n, in, Ci, El, B, Wk, bias, Co, out);
    if (Co % 32 == 0) return launch_conv3_tma_t<32, 8, RELU>(n, in, Ci, El, B, Wk, bias, Co, out);
    return launch_conv3_tma_t<16, 8, RELU>(n, in, Ci, El, B, Wk, bias, Co, out);
  }
  if (taps == 27 && n->tc) {  // tensor memory accumulators; columns per CTA: 64, 32 or 16
    const int B = (int)(nvox / ((long long)El * El * El));
    if (Co % 64 == 0) return launch_conv3_tc_t<64, 4, RELU>(n, in, Ci, El, B, Wk, bias, Co, out);
    if (Co % 32 == 0) return launch_conv3_tc_t<32, 4, RELU>(n, in, Ci, El, B, Wk, bias, Co, out);
    return launch_conv3_tc_t<16, 4, RELU>(n, in, Ci, El, B, Wk, bias, Co, out);
  }
  if (taps == 27) {  // brick-tiled direct convolution; columns per CTA: 32 or 16
    const int B = (int)(nvox / ((long long)El * El * El));
    if (Co % 32 == 0) return launch_conv3_t<32, RELU>(n, in, Ci, El, B, Wk, bias, Co, out);
    return launch_conv3_t<16, RELU>(n, in, Ci, El, B, Wk, bias, Co, out);
  }
  const int BN = tile_n(Co);
  dim3 grid(nb(nvox, TM), Co / BN);
  cudaStream_t s = n->stream;
  switch (BN) {
    case 64: k_conv<64, RELU><<<grid, 128, 0, s>>>(in, Ci, El, nvox, taps, Wk, bias, Co, out); break;
    case 32: k_conv<32, RELU><<<grid, 128, 0, s>>>(in, Ci, El, nvox, taps, Wk, bias, Co, out); break;
    case 16: k_conv<16, RELU><<<grid, 128, 0, s>>>(in, Ci, El, nvox, taps, Wk, bias, Co, out); break;
    default: set_error("net: unsupported channel count"); return TLB_ERR_ARG;
  }
  NET_LAUNCHED(n, "k_conv");
  return TLB_OK;
}

// out = sum of the nsplit rows of part ([nsplit][n]; overwritten).
tlb_status sum_splits(Net* n, float* part, int nsplit, long long nn, float* out) {
  int step = 1;
  if (nsplit > SPLIT_GROUP) {
    const unsigned groups = (unsigned)((nsplit + SPLIT_GROUP - 1) / SPLIT_GROUP);
    k_sum_groups<<<dim3(nb(nn, 128), groups), 128, 0, n->stream>>>(part, nsplit, nn);
    NET_LAUNCHED(n, "k_sum_groups");
    step = SPLIT_GROUP;
  }
  k_sum_splits<<<nb(nn, 64), 64, 0, n->stream>>>(part, nsplit, nn, step, out);
  NET_LAUNCHED(n, "k_sum_splits");
  return TLB_OK;
}

template <int BN>
tlb_status launch_wgrad3_t(Net* n, const Conv& c, const bf16* in, int El, int B, const bf16* gz) {
  tlb_status st;
  const int nbr = ((El + BRX - 1) / BRX) * ((El + BRY - 1) / BRY) * ((El + BRZ - 1) / BRZ) * B;
  const int tiles = (c.co / BN) * (c.ci / 16);
  const int nsplit = std::max(1, std::min(nbr, std::min(512, (2 * 152 * 4 + tiles - 1) / tiles)));
  constexpr int sm = wgrad3_smem<BN>();
  float* part = n->at<float>(n->o_part);
  TLB_CUDA(cudaFuncSetAttribute(k_wgrad3<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  k_wgrad3<BN><<<dim3(nsplit, c.co / BN, c.ci / 16), 128, sm, n->stream>>>(in, c.ci, El, B, gz, c.co, part);
  NET_LAUNCHED(n, "k_wgrad3");
  float* g = n->at<float>(n->o_grad);
  // weight gradient: sums over the CTAs' partials [27 * Ci][Co]
  const long long nw = 27ll * c.ci * c.co;
  if ((st = sum_splits(n, part, nsplit, nw, g + c.w)) != TLB_OK) return st;
  // bias gradient: column sums of gz over fixed voxel ranges, then over the ranges
  const long long V = (long long)B * El * El * El;
  const int nbs = (int)std::min<long long>(512, (V + 255) / 256);
  const long long chunk = (V + nbs - 1) / nbs;
  k_colsum<<<nbs, 256, 0, n->stream>>>(gz, V, c.co, chunk, part);
  NET_LAUNCHED(n, "k_colsum");
  if ((st = sum_splits(n, part, nbs, c.co, g + c.b)) != TLB_OK) return st;
  return TLB_OK;
}

tlb_status launch_wgrad(Net* n, const Conv& c, const bf16* in, int El, long long nvox, const bf16* gz) {
  if (c.taps == 27) {
    const int B = (int)(nvox / ((long long)El * El * El));
    if (c.co % 32 == 0) return launch_wgrad3_t<32>(n, c, in, El, B, gz);
    return launch_wgrad3_t<16>(n, c, in, El, B, gz);
  }
  const int BN = tile_n(c.co);
  const int M = c.taps * c.ci + 1;
  const int mt = (M + TM - 1) / TM, ntile = c.co / BN;
  long long splits = std::max(1LL, std::min(512LL, (long long)(2 * 152 * 4) / (mt * ntile)));
  long long vchunk = (nvox + splits - 1) / splits;
  vchunk = (vchunk + TK - 1) / TK * TK;
  splits = (nvox + vchunk - 1) / vchunk;
  dim3 grid(mt, ntile, (unsigned)splits);
  float* part = n->at<float>(n->o_part);
  cudaStream_t s = n->stream;
  switch (BN) {
    case 64: k_wgrad<64><<<grid, 128, 0, s>>>(in, c.ci, El, nvox, c.taps, gz, c.co, vchunk, part); break;
    case 32: k_wgrad<32><<<grid, 128, 0, s>>>(in, c.ci, El, nvox, c.taps, gz, c.co, vchunk, part); break;
    case 16: k_wgrad<16><<<grid, 128, 0, s>>>(in, c.ci, El, nvox, c.taps, gz, c.co, vchunk, part); break;
    default: set_error("net: unsupported channel count"); return TLB_ERR_ARG;
  }
  NET_LAUNCHED(n, "k_wgrad");
  float* g = n->at<float>(n->o_grad);
  k_wgrad_reduce<<<nb((long long)M * c.co, 256), 256, 0, s>>>(part, (int)splits, M, c.co, g + c.w, g + c.b);
  NET_LAUNCHED(n, "k_wgrad_reduce");
  return TLB_OK;
}

tlb_status refresh_weights(Net* n) {
  const float* th = n->at<float>(n->o_theta);
  for (const Conv& c : n->convs) {
    k_weights<<<nb((long long)c.taps * c.ci * c.co, 256), 256, 0, n->stream>>>(
        th + c.w, c.taps, c.ci, c.co, n->at<bf16>(n->o_wf) + c.wf, n->at<bf16>(n->o_wd) + c.wd);
    NET_LAUNCHED(n, "k_weights");
  }
  return TLB_OK;
}

// Forward pass of B samples from the input tensor x (already in place).
tlb_status forward(Net* n, int B) {
  const int L = n->d.levels;
  bf16* A = n->at<bf16>(n->o_act);
  const bf16* Wf = n->at<bf16>(n->o_wf);
  const float* th = n->at<float>(n->o_theta);
  cudaStream_t s = n->stream;
  tlb_status st;
  size_t k = 0;
  const bf16* h = A + n->x.act;
  int hc = 16;
  for (int l = 0; l < L; ++l) {
    const int El = n->d.edge >> l;
    const long long V = n->vox(l, B);
    if (l > 0) {
      bf16* p = A + n->enc_p[l].act;
      k_pool_fwd<<<nb(V * hc / 8, 256), 256, 0, s>>>(h, El * 2, hc, V, p);
      NET_LAUNCHED(n, "k_pool_fwd");
      h = p;
    }
    const Conv& c1 = n->convs[k++];
    if ((st = launch_conv<true>(n, h, c1.ci, El, V, 27, Wf + c1.wf, th + c1.b, c1.co, A + n->enc_a[l].act)) != TLB_OK)
      return st;
    const Conv& c2 = n->convs[k++];
    if ((st = launch_conv<true>(n, A + n->enc_a[l].act, c2.ci, El, V, 27, Wf + c2.wf, th + c2.b, c2.co,
                                A + n->enc_e[l].act)) != TLB_OK)
      return st;
    h = A + n->enc_e[l].act;
    hc = c2.co;
  }
  const bf16* dprev = A + n->enc_e[L - 1].act;
  for (int l = L - 2; l >= 0; --l) {
    const int El = n->d.edge >> l;
    const long long V = n->vox(l, B);
    const int C1 = n->chan(l + 1), C2 = n->chan(l);
    bf16* cat = A + n->dec_cat[l].act;
    k_cat_fwd<<<nb(V * ((C1 + C2) / 8), 256), 256, 0, s>>>(dprev, C1, A + n->enc_e[l].act, C2, El, V, cat);
    NET_LAUNCHED(n, "k_cat_fwd");
    const Conv& c1 = n->convs[k++];
    if ((st = launch_conv<true>(n, cat, c1.ci, El, V, 27, Wf + c1.wf, th + c1.b, c1.co, A + n->dec_b[l].act)) != TLB_OK)
      return st;
    const Conv& c2 = n->convs[k++];
    if ((st = launch_conv<true>(n, A + n->dec_b[l].act, c2.ci, El, V, 27, Wf + c2.wf, th + c2.b, c2.co,
                                A + n->dec_d[l].act)) != TLB_OK)
      return st;
    dprev = A + n->dec_d[l].act;
  }
  const Conv& co = n->convs[k++];
  return launch_conv<false>(n, dprev, co.ci, n->d.edge, n->vox(0, B), 1, Wf + co.wf, th + co.b, YC,
                            n->at<float>(n->o_y));
}

// Backward of one conv whose output is `out` (post-relu, bf16) with
// gradient g_out (fp32): weight/bias gradients, and the input gradient
// (fp32, overwritten) when g_in is non-null.
tlb_status conv_bwd(Net* n, const Conv& c, const bf16* in, const bf16* out, const float* g_out, float* g_in, int B,
                    bool relu) {
  const int El = n->d.edge >> c.level;
  const long long V = n->vox(c.level, B);
  bf16* gz = n->at<bf16>(n->o_gz);
  if (relu) k_relu_bwd<<<nb(V * c.co / 8, 256), 256, 0, n->stream>>>(g_out, out, V * c.co, gz);
  else k_to_bf16<<<nb(V * c.co / 8, 256), 256, 0, n->stream>>>(g_out, V * c.co, gz);
  NET_LAUNCHED(n, "k_relu_bwd");
  tlb_status st = launch_wgrad(n, c, in, El, V, gz);
  if (st != TLB_OK || !g_in) return st;
  return launch_conv<false>(n, gz, c.co, El, V, c.taps, n->at<bf16>(n->o_wd) + c.wd, nullptr, c.ci, g_in);
}

// Backward pass of B samples, from gy (loss gradient of the output) to the
// parameter gradients.  Order: the output conv, the decoder from the finest
// level up (its input gradient feeds the skip connection and the coarser
// level), then the encoder from the coarsest level down (the pooling
// gradient feeds the finer level).
tlb_status backward(Net* n, int B) {
  const int L = n->d.levels;
  bf16* A = n->at<bf16>(n->o_act);
  float* G = n->at<float>(n->o_grad_act);
  cudaStream_t s = n->stream;
  TLB_CUDA(cudaMemsetAsync(G, 0, n->n_gact * 4, s));
  tlb_status st;
  int k = (int)n->convs.size() - 1;
  const Ten& d0 = n->dec_d[0];
  if ((st = conv_bwd(n, n->convs[k--], A + d0.act, nullptr, n->at<float>(n->o_gy), G + d0.grad, B, false)) != TLB_OK)
    return st;
  for (int l = 0; l <= L - 2; ++l) {
    const Conv& c2 = n->convs[k--];
    const Conv& c1 = n->convs[k--];
    const int C1 = n->chan(l + 1), C2 = n->chan(l);
    const long long V = n->vox(l, B);
    const int El = n->d.edge >> l;
    if ((st = conv_bwd(n, c2, A + n->dec_b[l].act, A + n->dec_d[l].act, G + n->dec_d[l].grad, G + n->dec_b[l].grad,
                       B, true)) != TLB_OK)
      return st;
    if ((st = conv_bwd(n, c1, A + n->dec_cat[l].act, A + n->dec_b[l].act, G + n->dec_b[l].grad,
                       G + n->dec_cat[l].grad, B, true)) != TLB_OK)
      return st;
    k_cat_bwd_skip<<<nb(V * C2 / 4, 256), 256, 0, s>>>(G + n->dec_cat[l].grad, C1, C2, V, G + n->enc_e[l].grad);
    NET_LAUNCHED(n, "k_cat_bwd_skip");
    const Ten& coarse = (l + 1 <= L - 2) ? n->dec_d[l + 1] : n->enc_e[L - 1];
    k_cat_bwd_up<<<nb(n->vox(l + 1, B) * C1 / 4, 256), 256, 0, s>>>(G + n->dec_cat[l].grad, C1, C2, El,
                                                                 n->vox(l + 1, B), G + coarse.grad);
    NET_LAUNCHED(n, "k_cat_bwd_up");
  }
  for (int l = L - 1; l >= 0; --l) {
    const Conv& c2 = n->convs[k--];
    const Conv& c1 = n->convs[k--];
    if ((st = conv_bwd(n, c2, A + n->enc_a[l].act, A + n->enc_e[l].act, G + n->enc_e[l].grad, G + n->enc_a[l].grad,
                       B, true)) != TLB_OK)
      return st;
    const bf16* in = l > 0 ? A + n->enc_p[l].act : A + n->x.act;
    float* gin = l > 0 ? G + n->enc_p[l].grad : nullptr;
    if ((st = conv_bwd(n, c1, in, A + n->enc_a[l].act, G + n->enc_a[l].grad, gin, B, true)) != TLB_OK) return st;
    if (l > 0) {
      const long long Vf = n->vox(l - 1, B);
      k_pool_bwd<<<nb(Vf * c1.ci / 4, 256), 256, 0, s>>>(G + n->enc_p[l].grad, n->d.edge >> (l - 1), c1.ci, Vf,
                                                      G + n->enc_e[l - 1].grad);
      NET_LAUNCHED(n, "k_pool_bwd");
    }
  }
  return TLB_OK;
}

// Loss of the forward outputs of B samples against the targets; writes gy
// and returns the loss through tot (device, FP64).
tlb_status loss(Net* n, int B, const float* dphi, const float* dpsi, const float* X0, const float* off,
                const int* nnodes, double lambda, double* host_loss) {
  const long long V = n->vox(0, B), V1 = n->vox(0, 1);
  const int E = n->d.edge;
  cudaStream_t s = n->stream;
  double* part = n->at<double>(n->o_lpart);
  const unsigned nbf = nb(V, 256);
  long long* gfix = n->d.max_nodes > 0 ? n->at<long long>(n->o_gfix) : nullptr;
  k_loss_fields<<<nbf, 256, 0, s>>>(n->at<float>(n->o_y), dphi, dpsi, V, 1.0 / (double)V, n->at<float>(n->o_gy), gfix,
                                    part);
  NET_LAUNCHED(n, "k_loss_fields");
  long long ntot = 0;
  for (int b = 0; b < B; ++b) ntot += nnodes ? nnodes[b] : 0;
  unsigned nbn = 0;
  if (ntot > 0 && lambda != 0.0) {
    for (int b = 0; b < B; ++b) {
      if (nnodes[b] <= 0) continue;
      const unsigned k = nb(nnodes[b], 256);
      k_loss_nodes<<<k, 256, 0, s>>>(n->at<float>(n->o_y) + b * V1 * YC, X0 + (size_t)b * n->d.max_nodes * 3,
                                     off + (size_t)b * n->d.max_nodes * 3, nnodes[b], E, lambda / (3.0 * ntot),
                                     gfix + b * V1 * 3, part + nbf + nbn);
      NET_LAUNCHED(n, "k_loss_nodes");
      nbn += k;
    }
    if (nbn) {
      k_loss_fold<<<nbf, 256, 0, s>>>(gfix, V, n->at<float>(n->o_gy));
      NET_LAUNCHED(n, "k_loss_fold");
    }
  }
  double* tot = n->at<double>(n->o_misc);
  k_sum_parts<<<1, 256, 0, s>>>(part, (int)nbf, 1, tot);
  NET_LAUNCHED(n, "k_sum_parts");
  if (nbn) {
    k_sum_parts<<<1, 256, 0, s>>>(part + nbf, (int)nbn, 1, tot + 1);
    NET_LAUNCHED(n, "k_sum_parts");
  }
  double h[2] = {0, 0};
  TLB_CUDA(cudaMemcpyAsync(h, tot, (nbn ? 2 : 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  TLB_CUDA(cudaStreamSynchronize(s));
  if (host_loss) *host_loss = h[0] / (double)V + (nbn ? lambda * h[1] / (3.0 * ntot) : 0.0);
  return TLB_OK;
}

}  // namespace

extern "C" {

tlb_status tlb_net_param_count(const tlb_net_desc* desc, size_t* n) {
  tlb_status s = check_desc(desc);
  if (s != TLB_OK) return s;
  if (!n) { set_error("n is NULL"); return TLB_ERR_ARG; }
  Net net;
  net.d = *desc;
  plan(net);
  *n = net.nparam;
  return TLB_OK;
}

tlb_status tlb_net_state_bytes(const tlb_net_desc* desc, size_t* bytes) {
  tlb_status s = check_desc(desc);
  if (s != TLB_OK) return s;
  if (!bytes) { set_error("bytes is NULL"); return TLB_ERR_ARG; }
  Net net;
  net.d = *desc;
  plan(net);
  *bytes = net.bytes;
  return TLB_OK;
}

tlb_status tlb_net_create(const tlb_net_desc* desc, void* arena, size_t bytes, void* cuda_stream, void** net_out) {
  tlb_status s = check_desc(desc);
  if (s != TLB_OK) return s;
  if (!arena || !net_out) { set_error("arena and net_out must be non-NULL"); return TLB_ERR_ARG; }
  if (((uintptr_t)arena) & 255) { set_error("arena must be 256-byte aligned"); return TLB_ERR_ARG; }
  Net* n = new Net();
  n->d = *desc;
  plan(*n);
  if (bytes < n->bytes) {
    set_error("net arena too small: need " + std::to_string(n->bytes) + " bytes");
    delete n;
    return TLB_ERR_ALLOC;
  }
  n->base = (char*)arena;
  n->stream = (cudaStream_t)cuda_stream;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (n->nsm <= 0) n->nsm = 1;
  }
  s = cuda_check(cudaMemsetAsync(n->base, 0, n->bytes, n->stream), "memset net arena");
  if (s == TLB_OK) s = cuda_check(cudaStreamSynchronize(n->stream), "net create");
  if (s != TLB_OK) { delete n; return s; }
  *net_out = n;
  return TLB_OK;
}

tlb_status tlb_net_set_params(void* net, const float* host, size_t count) {
  Net* n = (Net*)net;
  if (!n || !host) { set_error("net/host is NULL"); return TLB_ERR_ARG; }
  if (count != n->nparam) { set_error("net_set_params: count differs from tlb_net_param_count"); return TLB_ERR_ARG; }
  TLB_CUDA(cudaMemcpyAsync(n->at<float>(n->o_theta), host, count * 4, cudaMemcpyHostToDevice, n->stream));
  TLB_CUDA(cudaMemsetAsync(n->at<float>(n->o_m), 0, count * 4, n->stream));
  TLB_CUDA(cudaMemsetAsync(n->at<float>(n->o_v), 0, count * 4, n->stream));
  n->adam_t = 0;
  n->launches = 0;
  tlb_status s = refresh_weights(n);
  if (s != TLB_OK) return s;
  TLB_CUDA(cudaStreamSynchronize(n->stream));
  return TLB_OK;
}

static tlb_status copy_out(Net* n, size_t off, float* host, size_t count) {
  if (!host) { set_error("host is NULL"); return TLB_ERR_ARG; }
  if (count != n->nparam) { set_error("net: count differs from tlb_net_param_count"); return TLB_ERR_ARG; }
  TLB_CUDA(cudaMemcpyAsync(host, n->at<float>(off), count * 4, cudaMemcpyDeviceToHost, n->stream));
  TLB_CUDA(cudaStreamSynchronize(n->stream));
  return TLB_OK;
}

tlb_status tlb_net_get_params(void* net, float* host, size_t count) {
  Net* n = (Net*)net;
  if (!n) { set_error("net is NULL"); return TLB_ERR_ARG; }
  return copy_out(n, n->o_theta, host, count);
}

tlb_status tlb_net_get_grads(void* net, float* host, size_t count) {
  Net* n = (Net*)net;
  if (!n) { set_error("net is NULL"); return TLB_ERR_ARG; }
  return copy_out(n, n->o_grad, host, count);
}

static tlb_status take_input(Net* n, const void* x_dev, int batch) {
  if (!x_dev) { set_error("x is NULL"); return TLB_ERR_ARG; }
  if (batch < 1 || batch > n->d.max_batch) { set_error("net: batch must be 1..max_batch"); return TLB_ERR_ARG; }
  TLB_CUDA(cudaMemcpyAsync(n->at<bf16>(n->o_act) + n->x.act, x_dev, (size_t)n->vox(0, batch) * 16 * 2,
                           cudaMemcpyDeviceToDevice, n->stream));
  return TLB_OK;
}

// The status word the tensor-core kernels set when a wait gave up: read
// (synchronising the stream) and cleared.
static tlb_status read_status(Net* n, unsigned* out) {
  unsigned h = 0;
  TLB_CUDA(cudaMemcpyAsync(&h, n->status(), 4, cudaMemcpyDeviceToHost, n->stream));
  TLB_CUDA(cudaStreamSynchronize(n->stream));
  if (h) TLB_CUDA(cudaMemsetAsync(n->status(), 0, 4, n->stream));
  if (out) *out = h;
  if (h) {
    set_error("net: a tensor-core wait gave up (status " + std::to_string(h) + ")");
    return TLB_ERR_CUDA;
  }
  return TLB_OK;
}

tlb_status tlb_net_status(void* net, unsigned* status) {
  Net* n = (Net*)net;
  if (!n) { set_error("net is NULL"); return TLB_ERR_ARG; }
  return read_status(n, status);
}

tlb_status tlb_net_set_tcgen05(void* net, int on) {
  Net* n = (Net*)net;
  if (!n) { set_error("net is NULL"); return TLB_ERR_ARG; }
  if (on < 0 || on > 2) { set_error("net_set_tcgen05: 0, 1 or 2"); return TLB_ERR_ARG; }
  n->tc = on;
  return TLB_OK;
}

tlb_status tlb_net_forward(void* net, const void* x_dev, int batch, float* y_dev) {
  Net* n = (Net*)net;
  if (!n) { set_error("net is NULL"); return TLB_ERR_ARG; }
  n->launches = 0;
  tlb_status s = take_input(n, x_dev, batch);
  if (s == TLB_OK) s = forward(n, batch);
  if (s != TLB_OK) return s;
  if (y_dev)
    TLB_CUDA(cudaMemcpyAsync(y_dev, n->at<float>(n->o_y), (size_t)n->vox(0, batch) * YC * 4, cudaMemcpyDeviceToDevice,
                             n->stream));
  return TLB_OK;
}

tlb_status tlb_net_train_step(void* net, const void* x_dev, const float* dphi_dev, const float* dpsi_dev,
                              const float* X0_dev, const float* off_dev, const int* n_nodes, int batch,
                              double lambda, double lr, int update, double* loss_out) {
  Net* n = (Net*)net;
  if (!n || !dphi_dev || !dpsi_dev) { set_error("net/targets are NULL"); return TLB_ERR_ARG; }
  if (n_nodes) {
    for (int b = 0; b < batch; ++b)
      if (n_nodes[b] < 0 || n_nodes[b] > n->d.max_nodes) { set_error("net: n_nodes outside 0..max_nodes"); return TLB_ERR_ARG; }
    bool any = false;
    for (int b = 0; b < batch; ++b) any |= n_nodes[b] > 0;
    if (any && (!X0_dev || !off_dev)) { set_error("net: marker arrays are NULL"); return TLB_ERR_ARG; }
  }
  n->launches = 0;
  tlb_status s = take_input(n, x_dev, batch);
  if (s == TLB_OK) s = forward(n, batch);
  if (s == TLB_OK) s = loss(n, batch, dphi_dev, dpsi_dev, X0_dev, off_dev, n_nodes, lambda, loss_out);
  if (s == TLB_OK) s = backward(n, batch);
  if (s != TLB_OK || !update) return s;
  n->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - pow(0.9, (double)n->adam_t)), c2 = (float)(1.0 - pow(0.999, (double)n->adam_t));
  k_adam<<<nb((long long)n->nparam, 256), 256, 0, n->stream>>>(n->at<float>(n->o_theta), n->at<float>(n->o_grad),
                                                               n->at<float>(n->o_m), n->at<float>(n->o_v),
                                                               (long long)n->nparam, (float)lr, b1, b2, 1e-8f, c1, c2);
  NET_LAUNCHED(n, "k_adam");
  s = refresh_weights(n);
  if (s == TLB_OK && loss_out) s = read_status(n, nullptr);
  return s;
}

static tlb_status check_ctx(Net* n, Ctx* c) {
  if (!c) { set_error("ctx is NULL"); return TLB_ERR_ARG; }
  if (c->p.dim != 3 || c->nx != n->d.edge || c->ny != n->d.edge || c->nz != n->d.edge) {
    set_error("net: the context must be a 3D lattice of edge^3 cells");
    return TLB_ERR_ARG;
  }
  if (c->ts.real != 4) { set_error("net: the context must compute in FP32 (storage f32, f16 or bf16)"); return TLB_ERR_ARG; }
  if (!c->initialised) { set_error("net: the context is not initialised"); return TLB_ERR_STATE; }
  return TLB_OK;
}

tlb_status tlb_net_input(void* net, void* ctx, const double* feats, void* x_dev) {
  Net* n = (Net*)net;
  Ctx* c = (Ctx*)ctx;
  if (!n || !feats || !x_dev) { set_error("net/feats/x is NULL"); return TLB_ERR_ARG; }
  tlb_status s = check_ctx(n, c);
  if (s != TLB_OK) return s;
  k_make_input<<<nb(c->N, 256), 256, 0, n->stream>>>(c->ptr<float>(c->L.phi), c->ptr<float>(c->L.psi), c->N,
                                                     (float)feats[0], (float)feats[1], (float)feats[2],
                                                     (float)feats[3], (float)feats[4], (bf16*)x_dev);
  NET_LAUNCHED(n, "k_make_input");
  return TLB_OK;
}

tlb_status tlb_net_warm_start(void* net, void* ctx, const double* feats) {
  Net* n = (Net*)net;
  Ctx* c = (Ctx*)ctx;
  if (!n || !feats) { set_error("net/feats is NULL"); return TLB_ERR_ARG; }
  tlb_status s = check_ctx(n, c);
  if (s != TLB_OK) return s;
  if (c->t != 0) { set_error("net_warm_start: the context must hold its initial state (no step taken)"); return TLB_ERR_STATE; }
  if (c->ncap != 1) { set_error("net_warm_start: the context must hold exactly one capsule"); return TLB_ERR_ARG; }
  // scratch: marker displacements in the output-gradient buffer, 3 sums per
  // 128-marker block in the loss partials
  if (3ll * c->nn > n->vox(0, n->d.max_batch) * YC || 3ll * nb(c->nn, 128) > 1024) {
    set_error("net_warm_start: too many markers for this net's scratch");
    return TLB_ERR_ARG;
  }
  TLB_CUDA(cudaStreamSynchronize(c->stream));
  n->launches = 0;
  cudaStream_t st = n->stream;
  bf16* x = n->at<bf16>(n->o_act) + n->x.act;
  float* phi = c->ptr<float>(c->L.phi);
  float* psi = c->ptr<float>(c->L.psi);
  float* I = c->ptr<float>(c->L.I);
  k_make_input<<<nb(c->N, 256), 256, 0, st>>>(phi, psi, c->N, (float)feats[0], (float)feats[1], (float)feats[2],
                                              (float)feats[3], (float)feats[4], x);
  NET_LAUNCHED(n, "k_make_input");
  if ((s = forward(n, 1)) != TLB_OK) return s;
  const float* y = n->at<float>(n->o_y);
  double* part = n->at<double>(n->o_lpart);
  double* tot = n->at<double>(n->o_misc) + 8;  // [0..3] pass 1, [4..5] pass 2, [8..10] translation
  // markers: mean translation plus the normal part of the predicted
  // displacement, then scaled about their centroid back to the plain
  // start's enclosed volume
  float* D = n->at<float>(n->o_gy);
  const unsigned bn = nb(c->nn, 128);
  double* X = c->ptr<double>(c->L.X);
  double* vol = n->at<double>(n->o_misc) + 32;  // [0, 1] area, volume before; [2, 3] after; [4..6] centroid sums
  k_capsule_measures<<<1, 256, 0, st>>>(X, c->ptr<int>(c->L.E), c->ptr<int>(c->L.ecap), c->ne, c->NV, 1, vol);
  NET_LAUNCHED(n, "k_capsule_measures");
  k_ws_disp<<<bn, 128, 0, st>>>(X, c->nn, y, n->d.edge, D, part);
  NET_LAUNCHED(n, "k_ws_disp");
  k_sum_parts<<<1, 256, 0, st>>>(part, (int)bn, 3, tot + 8);
  NET_LAUNCHED(n, "k_sum_parts");
  k_ws_move<<<bn, 128, 0, st>>>(X, c->nn, D, c->ptr<float>(c->L.vn), tot + 8);
  NET_LAUNCHED(n, "k_ws_move");
  k_capsule_measures<<<1, 256, 0, st>>>(X, c->ptr<int>(c->L.E), c->ptr<int>(c->L.ecap), c->ne, c->NV, 1, vol + 2);
  NET_LAUNCHED(n, "k_capsule_measures");
  k_ws_centroid<<<bn, 128, 0, st>>>(X, c->nn, part);
  NET_LAUNCHED(n, "k_ws_centroid");
  k_sum_parts<<<1, 256, 0, st>>>(part, (int)bn, 3, vol + 4);
  NET_LAUNCHED(n, "k_sum_parts");
  k_ws_scale<<<bn, 128, 0, st>>>(X, c->nn, vol + 4, vol, vol + 2);
  NET_LAUNCHED(n, "k_ws_scale");
  TLB_CUDA(cudaStreamSynchronize(st));
  // psi follows the moved membrane: its profile I, shifted to the plain total
  if ((s = c->impl->profile_now(c)) != TLB_OK) return s;
  TLB_CUDA(cudaStreamSynchronize(c->stream));
  k_ws_sums1<<<256, 256, 0, st>>>(phi, psi, I, c->N, part);
  NET_LAUNCHED(n, "k_ws_sums1");
  k_sum_parts<<<1, 256, 0, st>>>(part, 256, 4, tot);
  NET_LAUNCHED(n, "k_sum_parts");
  k_ws_sums2<<<256, 256, 0, st>>>(phi, psi, I, y, c->N, tot, part);
  NET_LAUNCHED(n, "k_ws_sums2");
  k_sum_parts<<<1, 256, 0, st>>>(part, 256, 2, tot + 4);
  NET_LAUNCHED(n, "k_sum_parts");
  k_ws_fields<<<nb(c->N, 256), 256, 0, st>>>(c->ptr<float>(c->L.rho), phi, psi, I, y, c->N, tot, tot + 4);
  NET_LAUNCHED(n, "k_ws_fields");
  TLB_CUDA(cudaStreamSynchronize(st));
  if ((s = read_status(n, nullptr)) != TLB_OK) return s;
  return c->impl->init_from_moments(c);
}

long tlb_net_launch_count(void* net) {
  Net* n = (Net*)net;
  return n ? n->launches : 0;
}

void tlb_net_destroy(void* net) { delete (Net*)net; }

}  // extern "C"
