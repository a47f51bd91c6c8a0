// Shared device definitions of the GB300 ternary LB + IBM library.
//
// Internal geometry: every lattice is stored as nx * ny * nz cells with
// linear index (z*ny + y)*nx + x.  A 2D lattice of the paper (D2Q9, Sec. 3.1)
// is embedded as nx * 1 * ny: its y axis becomes the internal z axis, so the
// same plane-sweep kernels serve both; markers of a 2D ring are stored as
// (x, 0, y).  Walls, when present, bound the internal z axis.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tlb.h"

#define TLB_HD __host__ __device__ __forceinline__

// ------------------------------------------------------------ velocity sets
// D2Q9 in the order printed in Sec. 3.1, embedded in the internal (x, z) plane.
struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int DIM = 2;
  TLB_HD static constexpr int cx(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 2 || i == 6 || i == 7 ? -1 : 0);
  }
  TLB_HD static constexpr int cy(int) { return 0; }
  TLB_HD static constexpr int cz(int i) {
    return i == 3 || i == 5 || i == 7 ? 1 : (i == 4 || i == 6 || i == 8 ? -1 : 0);
  }
  TLB_HD static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  TLB_HD static constexpr int opp(int i) {
    return i == 0 ? 0 : (i == 1 ? 2 : i == 2 ? 1 : i == 3 ? 4 : i == 4 ? 3 : i == 5 ? 6 : i == 6 ? 5 : i == 7 ? 8 : 7);
  }
};

// D3Q19: rest; +x,-x,+y,-y,+z,-z (w = 1/18); then the edge velocities of the
// xy, xz and yz planes with sign pairs (+,+),(+,-),(-,+),(-,-) (w = 1/36).
struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int DIM = 3;
  TLB_HD static constexpr int comp(int i, int a) {
    // axis velocities
    return i == 0 ? 0
         : i <= 6 ? ((i - 1) / 2 == a ? ((i - 1) % 2 == 0 ? 1 : -1) : 0)
                  : edge(i - 7, a);
  }
  TLB_HD static constexpr int edge(int e, int a) {
    // e = 4*plane + signs; planes (0,1), (0,2), (1,2)
    return (a == pa(e / 4) ? ((e % 4) < 2 ? 1 : -1) : 0) + (a == pb(e / 4) ? ((e % 4) % 2 == 0 ? 1 : -1) : 0);
  }
  TLB_HD static constexpr int pa(int p) { return p == 2 ? 1 : 0; }
  TLB_HD static constexpr int pb(int p) { return p == 0 ? 1 : 2; }
  TLB_HD static constexpr int cx(int i) { return comp(i, 0); }
  TLB_HD static constexpr int cy(int i) { return comp(i, 1); }
  TLB_HD static constexpr int cz(int i) { return comp(i, 2); }
  TLB_HD static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
  TLB_HD static constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 6 ? (i % 2 == 1 ? i + 1 : i - 1) : 7 + 4 * ((i - 7) / 4) + (3 - (i - 7) % 4));
  }
};

// ------------------------------------------------------------ precisions
template <int MODE> struct Prec;
template <> struct Prec<TLB_F64> { using Real = double; using Store = double; using Rest = double; };
template <> struct Prec<TLB_F32> { using Real = float; using Store = float; using Rest = float; };
template <> struct Prec<TLB_F16> { using Real = float; using Store = __half; using Rest = float; };
template <> struct Prec<TLB_BF16> { using Real = float; using Store = __nv_bfloat16; using Rest = float; };

TLB_HD double to_real(double v) { return v; }
TLB_HD float to_real(float v) { return v; }
__device__ __forceinline__ float to_real(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_real(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class S> __device__ __forceinline__ S from_real(double v);
template <class S> __device__ __forceinline__ S from_real(float v);
template <> __device__ __forceinline__ double from_real<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_real<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_real<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_real<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Two consecutive Real values (one 8 or 16-byte load).
template <class R> struct R2Of;
template <> struct R2Of<float> { using T = float2; };
template <> struct R2Of<double> { using T = double2; };
template <class R> using R2 = typename R2Of<R>::T;

// Two adjacent cells' values stored together (one 4, 8 or 16-byte store;
// p is aligned to two elements), each rounded as from_real rounds it.
__device__ __forceinline__ void store_pair(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
__device__ __forceinline__ void store_pair(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void store_pair(__half* p, float a, float b) {
  *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
}
__device__ __forceinline__ void store_pair(__nv_bfloat16* p, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}

// ------------------------------------------------------------ geometry
struct Geo {
  int nx, ny, nz;
  int wall;        // walls at both ends of z
  long long N;     // cells
  long long P;     // plane stride of population / field arrays (>= N, padded)
  int P32;         // P as int: every population offset (3Q planes) fits 31 bits
};

// Cell (x, y, z) of linear index n < N (N < 2^31: every population offset
// fits 31 bits), by two 32-bit divisions.
__device__ __forceinline__ void cell_xyz(const Geo& G, long long n, int& x, int& y, int& z) {
  const unsigned un = (unsigned)n, t = un / (unsigned)G.nx, zz = t / (unsigned)G.ny;
  x = (int)(un - t * (unsigned)G.nx);
  y = (int)(t - zz * (unsigned)G.ny);
  z = (int)zz;
}

// Block coordinates of a launch.  Kernel bodies take them as an argument, so
// one body runs either as its own grid (the hardware block index) or as one
// virtual block of a batched persistent launch over many lattices.
struct Blk {
  int x, y, z;     // block index
  int gx, gy, gz;  // grid size in blocks
};
__device__ __forceinline__ Blk hw_blk() {
  return {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x, (int)gridDim.y, (int)gridDim.z};
}

TLB_HD int wrapc(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Population layout: `lo` holds 3Q-2 planes of Store -- f_0..f_{Q-1} stored
// as f_i - w_i, then g_1..g_{Q-1}, then h_1..h_{Q-1}; `rest` holds g_0, h_0 in
// the Rest type.  Plane k of `lo` starts at lo + k*P.
template <class L> TLB_HD int plane_f(int i) { return i; }
template <class L> TLB_HD int plane_g(int i) { return L::Q + i - 1; }
template <class L> TLB_HD int plane_h(int i) { return 2 * L::Q - 1 + i - 1; }

template <class Real>
struct CellMoments {
  Real drho;     // rho - 1 (sum of the stored deviations)
  Real j[3];     // sum_i c_i f_i
  Real phi, psi;
};

// Source of the populations arriving at cell (x, y, z): direction i comes
// from x - c_i (periodic wrap), or, across a wall, from the cell itself in
// direction opp(i) (halfway bounce-back).  The wrapped neighbour rows are
// computed once per cell, so each pulled population costs one add.
template <class L>
struct Nbr {
  int self;
  int row[3][3];  // [dz + 1][dy + 1]: (z + dz, y + dy) row start
  int xs[3];      // x - 1, x, x + 1 (wrapped)
  bool wlo, whi;  // cell touches the bottom / top wall

  __device__ __forceinline__ Nbr(const Geo& G, int x, int y, int z) {
    self = (z * G.ny + y) * G.nx + x;
    xs[0] = x == 0 ? G.nx - 1 : x - 1;
    xs[1] = x;
    xs[2] = x == G.nx - 1 ? 0 : x + 1;
    int ys[3] = {y == 0 ? G.ny - 1 : y - 1, y, y == G.ny - 1 ? 0 : y + 1};
    int zs[3] = {z == 0 ? G.nz - 1 : z - 1, z, z == G.nz - 1 ? 0 : z + 1};
    wlo = G.wall && z == 0;
    whi = G.wall && z == G.nz - 1;
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) row[dz][dy] = (zs[dz] * G.ny + ys[dy]) * G.nx;
  }
  // bounce-back applies to direction i at this cell
  __device__ __forceinline__ bool bounce(int i) const {
    return (L::cz(i) > 0 && wlo) || (L::cz(i) < 0 && whi);
  }
  __device__ __forceinline__ int src(int i) const {
    return bounce(i) ? self : row[1 - L::cz(i)][1 - L::cy(i)] + xs[1 - L::cx(i)];
  }
  // offset of the population of direction i arriving here, in a plane array
  // whose plane for direction i (no bounce) or opp(i) (bounce) is given
  __device__ __forceinline__ int off(int i, int plane_i, int plane_opp, int P32) const {
    return (bounce(i) ? plane_opp : plane_i) * P32 + src(i);
  }
};

// Pull of the populations arriving at cell (x, y, z): f_i(x) = f*_i(x - c_i);
// across a wall, halfway bounce-back returns f*_{opp(i)}(x).  Both the moment
// kernel and the collision kernel use this routine so they agree bit for bit.
template <class L, int MODE>
struct Pull {
  using Real = typename Prec<MODE>::Real;
  using Store = typename Prec<MODE>::Store;
  using Rest = typename Prec<MODE>::Rest;
  Real f[L::Q], g[L::Q], h[L::Q];  // f holds f_i - w_i

  __device__ __forceinline__ void load(const Store* __restrict__ lo, const Rest* __restrict__ rest,
                                       const Geo& G, int x, int y, int z) {
    const Nbr<L> nb(G, x, y, z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      f[i] = to_real(__ldg(lo + nb.off(i, plane_f<L>(i), plane_f<L>(L::opp(i)), G.P32)));
      if (i == 0) {
        g[0] = to_real(__ldg(rest + nb.self));
        h[0] = to_real(__ldg(rest + G.P32 + nb.self));
      } else {
        g[i] = to_real(__ldg(lo + nb.off(i, plane_g<L>(i), plane_g<L>(L::opp(i)), G.P32)));
        h[i] = to_real(__ldg(lo + nb.off(i, plane_h<L>(i), plane_h<L>(L::opp(i)), G.P32)));
      }
    }
  }

  // The rest populations are added last: g_0 and h_0 carry nearly all of
  // phi and psi, so the small moving populations are summed first at their
  // own scale and the sum is rounded once at the scale of phi (adding them
  // one by one to g_0 rounds each addition there: in FP32 that made the
  // force about 4 times noisier).
  __device__ __forceinline__ CellMoments<Real> moments() const {
    CellMoments<Real> m;
    Real r = 0, jx = 0, jy = 0, jz = 0, p = 0, s = 0;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
      r += f[i];
      if (L::cx(i)) jx += L::cx(i) > 0 ? f[i] : -f[i];
      if (L::cy(i)) jy += L::cy(i) > 0 ? f[i] : -f[i];
      if (L::cz(i)) jz += L::cz(i) > 0 ? f[i] : -f[i];
      p += g[i];
      s += h[i];
    }
    r += f[0];
    p += g[0];
    s += h[0];
    m.drho = r;
    m.j[0] = jx;
    m.j[1] = jy;
    m.j[2] = jz;
    m.phi = p;
    m.psi = s;
    return m;
  }
};

// Cells the membrane work of a step touches: the marker box of the step
// (cur[0..2] = floor(min X), cur[3..5] = -ceil(max X)) widened by `margin`
// cells, unwrapped; walls clamp z; at most one period per axis.
__device__ __forceinline__ void marker_box(const int* cur, int margin, const Geo& G, bool d2, int* lo, int* hi) {
  const int n[3] = {G.nx, G.ny, G.nz};
  for (int d = 0; d < 3; ++d) {
    int bl = cur[d] - margin, bh = -cur[3 + d] + margin;
    if (d == 1 && d2) { bl = 0; bh = 0; }
    if (d == 2 && G.wall) { bl = max(bl, 0); bh = min(bh, n[2] - 1); }
    if (bh - bl + 1 > n[d]) bh = bl + n[d] - 1;
    if (bh < bl) bh = bl;
    lo[d] = bl;
    hi[d] = bh;
  }
}

// Chemical potentials of App. A (eq. AppA) without the ideal-gas part of
// mu_rho; mu_psi' adds kappa_c (psi - I) (Sec. 3.1).  The density enters as
// drho = rho - 1 (and Lr as its Laplacian, which is the Laplacian of rho):
// with A = rho + phi - psi = 1 + a, A (A - 1)(A - 2) = a (a^2 - 1), the same
// polynomial written around the bulk value, so that a working-precision
// drho keeps its low bits (rho = 1 + drho would round them away).
template <class Real>
struct FEParams {
  Real k1, k2, k3, kc, a2;  // kappa_1..3, kappa_c, alpha^2
};
template <class Real>
__device__ __forceinline__ void chem_potentials(const FEParams<Real>& fe, Real drho, Real phi, Real psi,
                                                Real Lr, Real Lp, Real Ls, Real I, Real& mr,
                                                Real& mp, Real& ms) {
  const Real a = drho + phi - psi, b = drho - phi - psi;  // A - 1, B - 1
  Real tA = fe.k1 * Real(0.125) * a * (a * a - Real(1));
  Real tB = fe.k2 * Real(0.125) * b * (b * b - Real(1));
  Real q = Real(0.25) * fe.a2;
  Real kp = fe.k1 + fe.k2, km = fe.k2 - fe.k1;
  mr = tA + tB + q * (kp * (Ls - Lr) + km * Lp);
  mp = tA - tB + q * (km * (Lr - Ls) - kp * Lp);
  ms = -tA - tB + q * (kp * Lr - km * Lp - (kp + Real(4) * fe.k3) * Ls) +
       fe.k3 * psi * (psi - Real(1)) * (Real(2) * psi - Real(1)) + fe.kc * (psi - I);
}

// Explicitly rounded arithmetic (round to nearest, never contracted): the
// same expression then rounds the same way in every kernel it is inlined
// into, whatever the compiler's multiply-add contraction would choose there.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// ------------------------------------------------ moment storage (tau = 1)
// At tau = tau_phi = tau_psi = 1 with the exact difference method every
// post-collision population is an equilibrium (eq. EDF) of its cell:
// f*_i = f_i^eq(rho, w) with w = u + du, g*_i = g_i^eq(phi, Gamma_phi mu_phi,
// v), h*_i = h_i^eq(psi, Gamma_psi mu_psi', v) (eq. LBE at tau = 1).  The
// moment-storage scheme keeps these 11 values per cell instead of the 3Q
// populations; the pull of the next step rebuilds each population from the
// cell it streams from.  Plane order of the stored moments:
enum { M_DRHO = 0, M_W = 1, M_PHI = 4, M_GMP = 5, M_PSI = 6, M_GMS = 7, M_V = 8, M_COUNT = 11 };

// Four values of one cell side by side, so that a shared-memory ring of them
// is read with one 16-byte load (two in double precision) per cell.
template <class R>
struct alignas(4 * sizeof(R)) R4 {
  R x, y, z, w;
};

// The post-collision populations of one cell from its stored moments, with
// the explicitly rounded operations (see rmul), so the reconstruction in the
// pull, in the interpolation and in the materialised populations gives the
// same value.
template <class L, class Real>
struct EqCell {
  Real drho, rho, w[3], ww, ord[2], gm3[2], v[3], vv;
  // drho and w only (what f_i needs)
  __device__ __forceinline__ void load_f(const Real* __restrict__ M, int P32, int c) {
    drho = M[M_DRHO * P32 + c];
#pragma unroll
    for (int d = 0; d < 3; ++d) w[d] = M[(M_W + d) * P32 + c];
    rho = Real(1) + drho;
    ww = rfma(w[2], w[2], rfma(w[1], w[1], rmul(w[0], w[0])));
  }
  __device__ __forceinline__ void load(const Real* __restrict__ M, int P32, int c) {
    load_f(M, P32, c);
    ord[0] = M[M_PHI * P32 + c];
    ord[1] = M[M_PSI * P32 + c];
    gm3[0] = rmul(Real(3), M[M_GMP * P32 + c]);
    gm3[1] = rmul(Real(3), M[M_GMS * P32 + c]);
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = M[(M_V + d) * P32 + c];
    vv = rfma(v[2], v[2], rfma(v[1], v[1], rmul(v[0], v[0])));
  }
  // the same from three packed values: (drho, w), (phi, Gamma_phi mu_phi,
  // psi, Gamma_psi mu_psi'), (v, -)
  __device__ __forceinline__ void load3(const R4<Real>& A, const R4<Real>& B, const R4<Real>& C) {
    drho = A.x;
    w[0] = A.y;
    w[1] = A.z;
    w[2] = A.w;
    rho = Real(1) + drho;
    ww = rfma(w[2], w[2], rfma(w[1], w[1], rmul(w[0], w[0])));
    ord[0] = B.x;
    ord[1] = B.z;
    gm3[0] = rmul(Real(3), B.y);
    gm3[1] = rmul(Real(3), B.w);
    v[0] = C.x;
    v[1] = C.y;
    v[2] = C.z;
    vv = rfma(v[2], v[2], rfma(v[1], v[1], rmul(v[0], v[0])));
  }
  // f_i - w_i = w_i (drho + rho (3 c.w + 4.5 (c.w)^2 - 1.5 w^2))
  __device__ __forceinline__ Real f(int i) const {
    const Real cw = L::cx(i) * w[0] + L::cy(i) * w[1] + L::cz(i) * w[2];
    const Real p = rfma(rmul(Real(4.5), cw), cw, rfma(Real(3), cw, rmul(Real(-1.5), ww)));
    return rmul(Real(L::w(i)), rfma(rho, p, drho));
  }
  // g_i (s = 0) or h_i (s = 1): w_i (3 Gamma mu + ord p(c.v)) for i != 0; the
  // rest population closes the zeroth moment
  __device__ __forceinline__ Real o(int s, int i) const {
    if (i == 0)
      return radd(rfma(gm3[s], Real(L::w(0)) - Real(1), ord[s]), rmul(rmul(Real(-1.5 * L::w(0)), ord[s]), vv));
    const Real cv = L::cx(i) * v[0] + L::cy(i) * v[1] + L::cz(i) * v[2];
    const Real p = rfma(rmul(Real(4.5), cv), cv, rfma(Real(3), cv, rmul(Real(-1.5), vv)));
    return rmul(Real(L::w(i)), rfma(ord[s], p, gm3[s]));
  }
};

// Status flags written by kernels (bitwise OR into a device word).
enum { ST_NAN = 1, ST_MARKER_JUMP = 2, ST_TIMEOUT = 4, ST_OVERFLOW = 8 };
