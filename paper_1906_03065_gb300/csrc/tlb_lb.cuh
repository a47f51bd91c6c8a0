// Lattice Boltzmann kernels: moments, chemical potentials, the fused
// force + collision + streaming plane sweep, initial equilibria and the
// conversions used by read/write of populations.
#pragma once
#include <type_traits>

#include "tlb_common.cuh"

template <int MODE>
struct LBArgs {
  using Real = typename Prec<MODE>::Real;
  using Store = typename Prec<MODE>::Store;
  using Rest = typename Prec<MODE>::Rest;
  Geo G;
  const Store* lo_src;
  const Rest* rest_src;
  Store* lo_dst;
  Rest* rest_dst;
  Real* rho;        // rho - 1 (the deviation keeps its low bits in FP32)
  Real* phi;
  Real* psi;
  Real* jm;         // [3][P] j of the streamed populations, written by the
                    // moments for the tau = 1 collide (NULL otherwise)
  Real* mst;        // moment storage: [11][P] moments the tau = 1 collide
                    // stores in place of the populations (NULL otherwise)
  const Real* msrc; // moment storage: the moments the reconstructing pull reads
  const Real* I;
  const Real* fib;  // [3][P] immersed-boundary force density
  Real* ftot;       // [3][P] total force of the step (read by the interpolation)
  const unsigned char* bflag;  // per 4x4x4 brick: markers spread force into it
  int nbx, nby;                // brick grid (x, y)
  FEParams<Real> fe;
  Real om, om_phi, om_psi;  // 1/tau
  Real gphi, gpsi;          // Gamma_phi, Gamma_psi
  int zc;                   // planes per block along z
  int forcing;              // TLB_FORCE_EDM or TLB_FORCE_GUO
  unsigned* status;
};

// Asynchronous global -> shared copies of one element (cp.async, 4 or 8
// bytes): the copy runs while the thread computes; cp_async_wait_all blocks
// until every copy the thread issued has landed.
__device__ __forceinline__ void cp_async_elem(float* dst, const float* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* dst, const double* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------- moments
// rho - 1, phi, psi at every cell from the streamed populations (eq.
// MomentsDFs), and j for the tau = 1 collide.
template <class L, int MODE>
__device__ __forceinline__ void moments_body(const LBArgs<MODE>& a, const Blk& blk) {
  using Real = typename Prec<MODE>::Real;
  const Geo G = a.G;
  long long n = (long long)blk.x * blockDim.x + threadIdx.x;
  if (n >= G.N) return;
  int x, y, z;
  cell_xyz(G, n, x, y, z);
  Pull<L, MODE> p;
  p.load(a.lo_src, a.rest_src, G, x, y, z);
  CellMoments<Real> m = p.moments();
  a.rho[n] = m.drho;
  a.phi[n] = m.phi;
  a.psi[n] = m.psi;
  if (a.jm) {
    a.jm[n] = m.j[0];
    a.jm[G.P + n] = m.j[1];
    a.jm[2 * G.P + n] = m.j[2];
  }
}
template <class L, int MODE>
__global__ void __launch_bounds__(256) k_moments(const __grid_constant__ LBArgs<MODE> a) {
  moments_body<L, MODE>(a, hw_blk());
}

// Moments of the streamed populations, each rebuilt from the stored moments
// of the cell it streams from (across a wall: this cell's opposite
// direction, halfway bounce-back); summed as the population pull sums.
template <class L, int MODE>
__device__ __forceinline__ void moments_recon_body(const LBArgs<MODE>& a, const Blk& blk) {
  using Real = typename Prec<MODE>::Real;
  const Geo G = a.G;
  long long n = (long long)blk.x * blockDim.x + threadIdx.x;
  if (n >= G.N) return;
  int x, y, z;
  cell_xyz(G, n, x, y, z);
  const Nbr<L> nb(G, x, y, z);
  Pull<L, MODE> p;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int ii = nb.bounce(i) ? L::opp(i) : i;
    EqCell<L, Real> e;
    e.load(a.msrc, G.P32, nb.src(i));
    p.f[i] = e.f(ii);
    p.g[i] = e.o(0, ii);
    p.h[i] = e.o(1, ii);
  }
  CellMoments<Real> m = p.moments();
  a.rho[n] = m.drho;
  a.phi[n] = m.phi;
  a.psi[n] = m.psi;
  a.jm[n] = m.j[0];
  a.jm[G.P + n] = m.j[1];
  a.jm[2 * G.P + n] = m.j[2];
}
template <class L, int MODE>
__global__ void __launch_bounds__(256) k_moments_recon(const __grid_constant__ LBArgs<MODE> a) {
  moments_recon_body<L, MODE>(a, hw_blk());
}

// The same pull as a plane sweep: a TX x TY tile of columns walks a chunk of
// z planes; the stored moments of four planes (tile plus a halo of 1) sit in
// a shared-memory ring filled by asynchronous copies one plane ahead, so
// every stored moment is read once from memory and a cell's rebuild reads
// its 19 sources from shared memory, three 16-byte vectors each.  Same
// arithmetic and summation order as moments_recon_body.
template <class L, int MODE, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_moments_recon_tiled(const __grid_constant__ LBArgs<MODE> a) {
  using Real = typename Prec<MODE>::Real;
  constexpr bool D3 = L::DIM == 3;
  constexpr int HX = TX + 2, HY = D3 ? TY + 2 : 1, CELLS = HX * HY, NT = TX * TY;
  struct Cell {
    R4<Real> a, b, c;  // (drho, w), (phi, gmp, psi, gms), (v, -)
  };
  __shared__ Cell sM[4][CELLS];
  const Geo G = a.G;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX, tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * a.zc;
  const int z1 = min(z0 + a.zc, G.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < G.nx && y < G.ny;
  auto wrapn = [](int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
  };
  // plane p of the ring (planes beyond a wall are never read: the pull
  // bounces there, so they take the nearest plane)
  auto issue_plane = [&](int p) {
    const int slot = (p + 8) & 3;
    const int pz = G.wall ? min(max(p, 0), G.nz - 1) : wrapn(p, G.nz);
    for (int k = tid; k < CELLS; k += NT) {
      const int hx = k % HX, hy = k / HX;
      const int gx = wrapn(x0 - 1 + hx, G.nx);
      const int gy = D3 ? wrapn(y0 - 1 + hy, G.ny) : 0;
      const long long c = ((long long)pz * G.ny + gy) * G.nx + gx;
      Real* d[M_COUNT] = {&sM[slot][k].a.x, &sM[slot][k].a.y, &sM[slot][k].a.z, &sM[slot][k].a.w,
                          &sM[slot][k].b.x, &sM[slot][k].b.y, &sM[slot][k].b.z, &sM[slot][k].b.w,
                          &sM[slot][k].c.x, &sM[slot][k].c.y, &sM[slot][k].c.z};
      // (plane order of the stored moments: drho, w, phi, gmp, psi, gms, v)
#pragma unroll
      for (int f = 0; f < M_COUNT; ++f) cp_async_elem(d[f], a.msrc + (long long)f * G.P + c);
    }
    cp_async_commit();
  };
  for (int p = z0 - 1; p <= z0 + 1; ++p) issue_plane(p);
  cp_async_wait_all();
  __syncthreads();
  for (int zz = z0; zz < z1; ++zz) {
    // plane zz + 2 replaces plane zz - 2, which this iteration does not read
    if (zz + 2 <= z1) issue_plane(zz + 2);
    if (active) {
      const bool wlo = G.wall && zz == 0, whi = G.wall && zz == G.nz - 1;
      Pull<L, MODE> p;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const bool bounce = (L::cz(i) > 0 && wlo) || (L::cz(i) < 0 && whi);
        const int ii = bounce ? L::opp(i) : i;
        const int sz = bounce ? zz : zz - L::cz(i);
        const int hx = bounce ? tx + 1 : tx + 1 - L::cx(i);
        const int hy = D3 ? (bounce ? ty + 1 : ty + 1 - L::cy(i)) : 0;
        EqCell<L, Real> e;
        const Cell& src = sM[(sz + 8) & 3][hy * HX + hx];
        e.load3(src.a, src.b, src.c);
        p.f[i] = e.f(ii);
        p.g[i] = e.o(0, ii);
        p.h[i] = e.o(1, ii);
      }
      const CellMoments<Real> m = p.moments();
      const long long n = ((long long)zz * G.ny + y) * G.nx + x;
      a.rho[n] = m.drho;
      a.phi[n] = m.phi;
      a.psi[n] = m.psi;
      a.jm[n] = m.j[0];
      a.jm[G.P + n] = m.j[1];
      a.jm[2 * G.P + n] = m.j[2];
    }
    cp_async_wait_all();
    __syncthreads();
  }
}

// The populations a cell's stored moments stand for, written post-collision
// into the population buffers (for the readers of the population state).
template <class L, int MODE>
__global__ void k_materialize(Geo G, const typename Prec<MODE>::Real* M, typename Prec<MODE>::Store* lo,
                              typename Prec<MODE>::Rest* rest) {
  using Real = typename Prec<MODE>::Real;
  using Store = typename Prec<MODE>::Store;
  using Rest = typename Prec<MODE>::Rest;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= G.N) return;
  EqCell<L, Real> e;
  e.load(M, G.P32, (int)n);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    lo[(long long)plane_f<L>(i) * G.P + n] = from_real<Store>(e.f(i));
    if (i == 0) {
      rest[n] = from_real<Rest>(e.o(0, 0));
      rest[G.P + n] = from_real<Rest>(e.o(1, 0));
    } else {
      lo[(long long)plane_g<L>(i) * G.P + n] = from_real<Store>(e.o(0, i));
      lo[(long long)plane_h<L>(i) * G.P + n] = from_real<Store>(e.o(1, i));
    }
  }
}

// Second-order polynomial of the equilibria: 3 c.u + 4.5 (c.u)^2 - 1.5 u^2.
template <class Real>
__device__ __forceinline__ Real eq_poly(Real cu, Real uu) {
  return Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * uu;
}

// ------------------------------------------------- fused collide + stream
// One block owns a TX x TY tile of (x, y) columns and sweeps a chunk of z
// planes.  Shared memory holds a 5-plane ring of the moment fields rho - 1,
// phi, psi (halo 2,
// written by k_moments; halo reads are served by L2) and a 3-plane ring of
// the chemical potentials (halo 1), so each cell's radius-2 dependency (mu
// needs the Laplacian of the moments, the force needs the gradient of mu) is
// served on chip.
// Pressure tensor of App. A without its ideal-gas part rho cs^2 delta (the
// force form grad(rho cs^2) - div p needs only the rest), in the variables
// rho, phi, psi with the mixing coefficients k_rr = k_ff = (k1 + k2)/4,
// k_ss = (k1 + k2 + 4 k3)/4, k_rf = -k_fs = (k1 - k2)/4, k_rs = -(k1 + k2)/4:
//   p'_ab = p'_b delta_ab + alpha^2 sum_mn k_mn [d_a m d_b n - delta_ab
//           ((1/2) grad m . grad n + m lap n)],
// with the bulk pressure of eq. PressureV2 (the ideal part dropped),
// p'_b = rho mu_rho^b + phi mu_phi^b + psi mu_psi^b - f_b and f_b = sum_m
// kappa_m/2 C_m^2 (1 - C_m)^2 = kappa1/32 (1 - a^2)^2 + kappa2/32 (1 - b^2)^2
// + kappa3/2 psi^2 (1 - psi)^2 (a = A - 1, b = B - 1 as in chem_potentials).
// Components xx, yy, zz, xy, xz, yz.  gr: the lattice gradients of rho - 1,
// phi, psi; lap: their Laplacians.
template <class Real>
__device__ __forceinline__ void pressure_tensor(const FEParams<Real>& fe, Real drho, Real phi, Real psi,
                                                const Real* lap, const Real (*gr)[3], Real* out) {
  const Real a = drho + phi - psi, b = drho - phi - psi;
  const Real tA = fe.k1 * Real(0.125) * a * (a * a - Real(1));
  const Real tB = fe.k2 * Real(0.125) * b * (b * b - Real(1));
  const Real ta = Real(1) - a * a, tb = Real(1) - b * b, tp = psi * (Real(1) - psi);
  const Real fb = fe.k1 * Real(1.0 / 32) * ta * ta + fe.k2 * Real(1.0 / 32) * tb * tb + fe.k3 * Real(0.5) * tp * tp;
  const Real rho = Real(1) + drho;
  const Real pb = rho * (tA + tB) + phi * (tA - tB) +
                  psi * (-tA - tB + fe.k3 * psi * (psi - Real(1)) * (Real(2) * psi - Real(1))) - fb;
  const Real kp = Real(0.25) * (fe.k1 + fe.k2), km = Real(0.25) * (fe.k1 - fe.k2);
  const Real K[3][3] = {{kp, km, -kp}, {km, kp, -km}, {-kp, -km, kp + fe.k3}};
  const Real val[3] = {rho, phi, psi};
  Real tr = pb;
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      const Real gg = gr[m][0] * gr[n][0] + gr[m][1] * gr[n][1] + gr[m][2] * gr[n][2];
      tr -= fe.a2 * K[m][n] * (Real(0.5) * gg + val[m] * lap[n]);
    }
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    Real t = ia[q] == ib[q] ? tr : Real(0);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int n = 0; n < 3; ++n) t += fe.a2 * K[m][n] * gr[m][ia[q]] * gr[n][ib[q]];
    out[q] = t;
  }
}

// Forms 5 and 6 are the collide at tau = tau_phi = tau_psi = 1 with the exact
// difference method: there every post-collision population is an
// equilibrium, f* = f^eq(rho, u + du), g* = g^eq(phi, mu_phi, v), h* =
// h^eq(psi, mu_psi', v) (eq. LBE with tau = 1), so the collide reads the
// moments rho - 1 and j that the moment pass wrote (summed in the same order
// as the pull of the general forms) and pulls no population: it only stores
// them.
template <int FORM> constexpr bool form_t1() { return FORM == 5 || FORM == 6 || FORM == 8 || FORM == 9; }
// forms 8 and 9: the tau = 1 collide with two x-adjacent cells per thread
template <int FORM> constexpr bool form_pair() { return FORM == 8 || FORM == 9; }

template <class L, int MODE, int TX, int TY, int FORM>
__device__ __forceinline__ void collide_gen_body(const LBArgs<MODE>& a, const Blk& blk) {
  constexpr bool PF = FORM == 1;  // the next population set prefetched
  constexpr bool T1 = form_t1<FORM>();
  // form 7: the force from the explicit pressure tensor (see pt_of)
  constexpr bool PT = FORM == 7;
  using Real = typename Prec<MODE>::Real;
  using Store = typename Prec<MODE>::Store;
  using Rest = typename Prec<MODE>::Rest;
  constexpr int Q = L::Q;
  constexpr bool D3 = L::DIM == 3;
  constexpr int HY = D3 ? 2 : 0;
  constexpr int MX = TX + 4, MY = TY + 2 * HY;
  constexpr int UX = TX + 2, UY = TY + (D3 ? 2 : 0);
  constexpr int NT = TX * TY;
  // per cell of the potentials' ring: mu~rho, mu_phi, mu_psi'; with the
  // pressure tensor: p_xx p_yy p_zz p_xy p_xz p_yz, kappa_c (psi - I),
  // mu_phi, mu_psi'
  constexpr int NMU = PT ? 9 : 3;
  constexpr int MUP = PT ? 7 : 1, MUS = PT ? 8 : 2;  // slots of mu_phi, mu_psi'
  __shared__ Real smom[5][3][MY * MX];
  __shared__ Real smu[3][NMU][UY * UX];

  const Geo G = a.G;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX, tid = threadIdx.x;
  const int x0 = blk.x * TX, y0 = blk.y * TY;
  const int z0 = blk.z * a.zc;
  const int z1 = min(z0 + a.zc, G.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < G.nx && y < G.ny;

  // wrap of a halo index: within two cells of the range except for tiles
  // wider than the lattice, which take the division
  auto modn = [](int v, int n) {
    if (v < 0) v += n;
    if (v >= n) v -= n;
    if (v < 0 || v >= n) {
      v %= n;
      if (v < 0) v += n;
    }
    return v;
  };
  auto plane_src = [&](int p) { return G.wall ? min(max(p, 0), G.nz - 1) : modn(p, G.nz); };

  auto load_mom = [&](int p) {
    const int slot = (p + 10) % 5;
    const long long zp = (long long)plane_src(p) * G.ny;
    for (int k = tid; k < MX * MY; k += NT) {
      int hx = k % MX, hy = k / MX;
      int gx = modn(x0 - 2 + hx, G.nx);
      int gy = D3 ? modn(y0 - HY + hy, G.ny) : 0;
      long long c = (zp + gy) * G.nx + gx;
      smom[slot][0][k] = a.rho[c];
      smom[slot][1][k] = a.phi[c];
      smom[slot][2][k] = a.psi[c];
    }
  };

  // chemical potentials of plane p on the tile plus a halo of 1
  auto compute_mu = [&](int p) {
    const int slot = (p + 9) % 3;
    if (G.wall && (p < 0 || p >= G.nz)) {  // mirror ghost: mu(-1) = mu(0), mu(nz) = mu(nz-1)
      const int src = (min(max(p, 0), G.nz - 1) + 9) % 3;
      for (int k = tid; k < UX * UY; k += NT)
        for (int q = 0; q < NMU; ++q) smu[slot][q][k] = smu[src][q][k];
      return;
    }
    const long long zp = (long long)modn(p, G.nz) * G.ny;  // periodic ghost planes wrap
    for (int k = tid; k < UX * UY; k += NT) {
      int ux = k % UX, uy = k / UX;
      int hx = ux + 1, hy = uy + (D3 ? 1 : 0);
      const int sc = (p + 10) % 5;
      const int cidx = hy * MX + hx;
      Real lap[3] = {0, 0, 0};
      Real cen[3] = {smom[sc][0][cidx], smom[sc][1][cidx], smom[sc][2][cidx]};
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int s = (p + L::cz(i) + 10) % 5;
        const int nb = (hy + L::cy(i)) * MX + hx + L::cx(i);
        const Real w = Real(L::w(i));
#pragma unroll
        for (int q = 0; q < 3; ++q) lap[q] += w * (smom[s][q][nb] - cen[q]);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) lap[q] *= Real(6);  // 2/cs^2
      int gx = modn(x0 - 1 + ux, G.nx);
      int gy = D3 ? modn(y0 - 1 + uy, G.ny) : 0;
      Real Iv = a.I[(zp + gy) * G.nx + gx];
      Real mr, mp, ms;
      chem_potentials<Real>(a.fe, cen[0], cen[1], cen[2], lap[0], lap[1], lap[2], Iv, mr, mp, ms);
      if constexpr (PT) {
        // gradients of rho - 1, phi, psi (radius 1, isotropic stencil)
        Real gr[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const int s = (p + L::cz(i) + 10) % 5;
          const int nb = (hy + L::cy(i)) * MX + hx + L::cx(i);
          const Real w = Real(L::w(i)) * Real(3);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const Real v = w * smom[s][q][nb];
            if (L::cx(i)) gr[q][0] += L::cx(i) > 0 ? v : -v;
            if (L::cy(i)) gr[q][1] += L::cy(i) > 0 ? v : -v;
            if (L::cz(i)) gr[q][2] += L::cz(i) > 0 ? v : -v;
          }
        }
        Real pt[6];
        pressure_tensor<Real>(a.fe, cen[0], cen[1], cen[2], lap, gr, pt);
#pragma unroll
        for (int q = 0; q < 6; ++q) smu[slot][q][k] = pt[q];
        smu[slot][6][k] = a.fe.kc * (cen[2] - Iv);
        smu[slot][MUP][k] = mp;
        smu[slot][MUS][k] = ms;
      } else {
        smu[slot][0][k] = mr;
        smu[slot][1][k] = mp;
        smu[slot][2][k] = ms;
      }
    }
  };

  // Collision of one cell.  rho, phi, psi come from the moment ring (k_moments
  // summed them in the same order as Pull::moments); the three population
  // sets are pulled, collided and stored one after another, so only one set
  // is live in registers at a time.
  auto collide = [&](int zz) {
    if (!active) return;
    const Nbr<L> nb(G, x, y, zz);
    const int n = nb.self;
    const int sm5 = (zz + 10) % 5;
    const int mc = (ty + HY) * MX + tx + 2;
    const Real drho_c = smom[sm5][0][mc], phi = smom[sm5][1][mc], psi = smom[sm5][2][mc];
    const Real rho = Real(1) + drho_c;
    // gradients of the potentials' ring entries (radius 1, isotropic
    // stencil; the 1/cs^2 is applied below)
    constexpr int NG = PT ? 7 : 3;
    Real gm[NG][3];
#pragma unroll
    for (int q = 0; q < NG; ++q) gm[q][0] = gm[q][1] = gm[q][2] = Real(0);
    const int ux = tx + 1, uy = ty + (D3 ? 1 : 0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int s = (zz + L::cz(i) + 9) % 3;
      const int nbi = (uy + L::cy(i)) * UX + ux + L::cx(i);
      const Real w = Real(L::w(i));
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        const Real v = w * smu[s][q][nbi];
        if (L::cx(i)) gm[q][0] += L::cx(i) > 0 ? v : -v;
        if (L::cy(i)) gm[q][1] += L::cy(i) > 0 ? v : -v;
        if (L::cz(i)) gm[q][2] += L::cz(i) > 0 ? v : -v;
      }
    }
    const int sc = (zz + 9) % 3;
    const int cc = uy * UX + ux;
    const Real mup = smu[sc][MUP][cc], mus = smu[sc][MUS][cc];
    // force (+ f_IB inside the bricks the markers spread into):
    //  potential form: f_FE = -rho grad mu~rho - phi grad mu_phi - psi grad mu_psi'
    //  pressure-tensor form: f_FE = -div p' - psi grad(kappa_c (psi - I)), p' the
    //  tensor of App. A without rho cs^2 (whose divergence cancels grad rho cs^2)
    const bool ib = a.bflag[((zz >> 2) * a.nby + (y >> 2)) * a.nbx + (x >> 2)] != 0;
    Real F[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if constexpr (PT) {
        // row d of the symmetric tensor: (xx, xy, xz), (xy, yy, yz), (xz, yz, zz)
        const int r0 = d == 0 ? 0 : (d == 1 ? 3 : 4), r1 = d == 0 ? 3 : (d == 1 ? 1 : 5),
                  r2 = d == 0 ? 4 : (d == 1 ? 5 : 2);
        F[d] = -Real(3) * (gm[r0][0] + gm[r1][1] + gm[r2][2] + psi * gm[6][d]);
      } else {
        F[d] = -Real(3) * (rho * gm[0][d] + phi * gm[1][d] + psi * gm[2][d]);
      }
      if (ib) F[d] += a.fib[d * G.P32 + n];
    }
    if (!D3) F[1] = 0;
    // pull of the order-parameter set `set` (0: g, 1: h) into v
    auto load_set = [&](int set, Real* v) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (i == 0) {
          v[0] = to_real(__ldg(a.rest_src + (set == 0 ? 0 : G.P32) + n));
        } else {
          const int o = set == 0 ? nb.off(i, plane_g<L>(i), plane_g<L>(L::opp(i)), G.P32)
                                 : nb.off(i, plane_h<L>(i), plane_h<L>(L::opp(i)), G.P32);
          v[i] = to_real(__ldg(a.lo_src + o));
        }
      }
    };
    // f: pull, first moment, BGK + exact difference method (eq. LBE) for f_i - w_i
    Real fv[T1 ? 1 : Q];
    Real drho = 0, jx = 0, jy = 0, jz = 0;
    // with PF the next set's loads are in flight while this one is computed
    Real nextv[PF ? Q : 1];
    if constexpr (T1) {
      drho = drho_c;
      jx = a.jm[n];
      jy = a.jm[G.P32 + n];
      jz = a.jm[2 * G.P32 + n];
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        fv[i] = to_real(__ldg(a.lo_src + nb.off(i, plane_f<L>(i), plane_f<L>(L::opp(i)), G.P32)));
      }
      if constexpr (PF) load_set(0, nextv);
#pragma unroll
      for (int i = 1; i < Q; ++i) {  // in the order of Pull::moments (rest last)
        drho += fv[i];
        if (L::cx(i)) jx += L::cx(i) > 0 ? fv[i] : -fv[i];
        if (L::cy(i)) jy += L::cy(i) > 0 ? fv[i] : -fv[i];
        if (L::cz(i)) jz += L::cz(i) > 0 ? fv[i] : -fv[i];
      }
      drho += fv[0];
    }
    const Real irho = Real(1) / rho;
    const Real j[3] = {jx, jy, jz};
    Real u[3], du[3], v[3], us[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      u[d] = j[d] * irho;
      du[d] = F[d] * irho;
      v[d] = u[d] + Real(0.5) * du[d];
      us[d] = u[d] + u[d] + du[d];  // u + (u + du)
    }
    const Real uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const Real vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const Real dus = du[0] * us[0] + du[1] * us[1] + du[2] * us[2];
    const Real om = a.om;
    if constexpr (T1) {
      if (a.mst) {
        // moment storage: the 11 values whose equilibria are this cell's
        // post-collision populations (see EqCell)
        Real* M = a.mst;
        M[M_DRHO * G.P32 + n] = drho;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          M[(M_W + d) * G.P32 + n] = radd(u[d], du[d]);
          M[(M_V + d) * G.P32 + n] = v[d];
        }
        M[M_PHI * G.P32 + n] = phi;
        M[M_GMP * G.P32 + n] = a.gphi * mup;
        M[M_PSI * G.P32 + n] = psi;
        M[M_GMS * G.P32 + n] = a.gpsi * mus;
        if (ib)
#pragma unroll
          for (int d = 0; d < 3; ++d) a.ftot[d * G.P32 + n] = F[d];
        if (!(rho == rho) || !(phi == phi) || !(psi == psi)) atomicOr(a.status, (unsigned)ST_NAN);
        return;
      }
      // f* = f^eq(rho, u + du), written as w [drho + rho p(u)] + w rho dP with
      // the explicitly rounded operations (see rmul)
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const Real w = Real(L::w(i));
        const Real wrho = rmul(rho, w);
        const Real cu = L::cx(i) * u[0] + L::cy(i) * u[1] + L::cz(i) * u[2];
        const Real cdu = L::cx(i) * du[0] + L::cy(i) * du[1] + L::cz(i) * du[2];
        const Real cus = L::cx(i) * us[0] + L::cy(i) * us[1] + L::cz(i) * us[2];
        const Real pu = rfma(rmul(Real(4.5), cu), cu, rfma(Real(3), cu, rmul(Real(-1.5), uu)));
        const Real dP = rfma(rmul(Real(4.5), cdu), cus, rfma(Real(3), cdu, rmul(Real(-1.5), dus)));
        const Real fn = rfma(wrho, dP, rmul(w, rfma(rho, pu, drho)));
        a.lo_dst[plane_f<L>(i) * G.P32 + n] = from_real<Store>(fn);
      }
    } else if (a.forcing == TLB_FORCE_GUO) {
      // Guo forcing: BGK towards f^eq(rho, v) plus (1 - om/2) w_i [3 (c_i - v) + 9 (c_i.v) c_i] . F
      const Real vF = v[0] * F[0] + v[1] * F[1] + v[2] * F[2];
      const Real sc = Real(1) - Real(0.5) * om;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const Real w = Real(L::w(i));
        const Real cv = L::cx(i) * v[0] + L::cy(i) * v[1] + L::cz(i) * v[2];
        const Real cF = L::cx(i) * F[0] + L::cy(i) * F[1] + L::cz(i) * F[2];
        const Real fn = (Real(1) - om) * fv[i] + om * w * (drho + rho * eq_poly(cv, vv)) +
                        sc * w * (Real(3) * (cF - vF) + Real(9) * cv * cF);
        a.lo_dst[plane_f<L>(i) * G.P32 + n] = from_real<Store>(fn);
      }
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const Real w = Real(L::w(i));
        const Real cu = L::cx(i) * u[0] + L::cy(i) * u[1] + L::cz(i) * u[2];
        const Real cdu = L::cx(i) * du[0] + L::cy(i) * du[1] + L::cz(i) * du[2];
        const Real cus = L::cx(i) * us[0] + L::cy(i) * us[1] + L::cz(i) * us[2];
        const Real dP = Real(3) * cdu + Real(4.5) * cdu * cus - Real(1.5) * dus;
        const Real fn = (Real(1) - om) * fv[i] + om * w * (drho + rho * eq_poly(cu, uu)) + w * rho * dP;
        a.lo_dst[plane_f<L>(i) * G.P32 + n] = from_real<Store>(fn);
      }
    }
    // g and h: BGK towards the order-parameter equilibria at v (eq. EDF); the
    // rest population closes the zeroth moment
    const Real w0 = Real(L::w(0));
#pragma unroll
    for (int set = 0; set < 2; ++set) {
      const Real om_s = set == 0 ? a.om_phi : a.om_psi;
      const Real Gm = set == 0 ? a.gphi * mup : a.gpsi * mus;
      const Real ord = set == 0 ? phi : psi;
      Real gv[T1 ? 1 : Q];
      if constexpr (T1) {
        // (om_s = 1: the post-collision set is the equilibrium)
      } else if constexpr (PF) {
#pragma unroll
        for (int i = 0; i < Q; ++i) gv[i] = nextv[i];
        if (set == 0) load_set(1, nextv);
      } else {
        load_set(set, gv);
      }
      if constexpr (T1) {
        // g* = g^eq(ord, mu, v) (om_s = 1), explicitly rounded (see rmul)
        const Real g3 = rmul(Real(3), Gm);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const Real w = Real(L::w(i));
          const Real cv = L::cx(i) * v[0] + L::cy(i) * v[1] + L::cz(i) * v[2];
          const Real pv = rfma(rmul(Real(4.5), cv), cv, rfma(Real(3), cv, rmul(Real(-1.5), vv)));
          const int pp = set == 0 ? plane_g<L>(i) : plane_h<L>(i);
          a.lo_dst[pp * G.P32 + n] = from_real<Store>(rmul(w, rfma(ord, pv, g3)));
        }
        // ord - 3 Gm (1 - w0) - 1.5 w0 ord v^2
        const Real ge0 = radd(rfma(g3, w0 - Real(1), ord), rmul(rmul(Real(-1.5) * w0, ord), vv));
        a.rest_dst[(set == 0 ? 0 : G.P32) + n] = from_real<Rest>(ge0);
      } else {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const Real w = Real(L::w(i));
          const Real cv = L::cx(i) * v[0] + L::cy(i) * v[1] + L::cz(i) * v[2];
          const Real pv = Real(3) * cv + Real(4.5) * cv * cv - Real(1.5) * vv;
          const Real ge = w * (Real(3) * Gm + ord * pv);
          const int pp = set == 0 ? plane_g<L>(i) : plane_h<L>(i);
          a.lo_dst[pp * G.P32 + n] = from_real<Store>((Real(1) - om_s) * gv[i] + om_s * ge);
        }
        const Real ge0 = ord - Real(3) * Gm * (Real(1) - w0) - Real(1.5) * w0 * ord * vv;
        a.rest_dst[(set == 0 ? 0 : G.P32) + n] = from_real<Rest>((Real(1) - om_s) * gv[0] + om_s * ge0);
      }
    }
    if (ib)
#pragma unroll
      for (int d = 0; d < 3; ++d) a.ftot[d * G.P32 + n] = F[d];
    if (!(rho == rho) || !(phi == phi) || !(psi == psi)) atomicOr(a.status, (unsigned)ST_NAN);
  };

  // prologue: moments z0-2 .. z0+1, potentials z0 then z0-1 (a wall ghost
  // copies its neighbour, so the real plane comes first)
  for (int p = z0 - 2; p <= z0 + 1; ++p) load_mom(p);
  __syncthreads();
  compute_mu(z0);
  __syncthreads();
  compute_mu(z0 - 1);
  __syncthreads();
  for (int zz = z0; zz < z1; ++zz) {
    load_mom(zz + 2);
    __syncthreads();
    compute_mu(zz + 1);
    __syncthreads();
    collide(zz);
    __syncthreads();
  }
}

// The collide of forms 5 and 6 (tau = tau_phi = tau_psi = 1, exact
// difference method): every post-collision population is an equilibrium of
// the cell's moments, so nothing is pulled; the kernel is a plane sweep over
// the moment fields that stores 3Q populations per cell (or, with moment
// storage, the 11 moments).  Per plane: the ring plane three ahead (rho - 1,
// phi, psi and I, tile plus a halo of 2) is copied asynchronously into the
// 5-plane ring while the potentials of the next plane and the collision of
// this one are computed.  The equilibria of opposite velocities share their
// even part, and g and h share the velocity polynomial; all rounded
// explicitly (see rmul), so every kernel it is inlined into computes the
// same values.
template <class L, int MODE, int TX, int TY, int FORM>
__device__ __forceinline__ void collide_t1_body(const LBArgs<MODE>& a, const Blk& blk) {
  using Real = typename Prec<MODE>::Real;
  using Store = typename Prec<MODE>::Store;
  using Rest = typename Prec<MODE>::Rest;
  constexpr int Q = L::Q;
  constexpr bool D3 = L::DIM == 3;
  constexpr int HY = D3 ? 2 : 0;
  constexpr int MX = TX + 4, MY = TY + 2 * HY;
  constexpr int UX = TX + 2, UY = TY + (D3 ? 2 : 0);
  // cells per thread: two x-adjacent cells in the pair forms (8, 9)
  constexpr int NC = form_pair<FORM>() ? 2 : 1;
  constexpr int NT = TX / NC * TY;
  __shared__ R4<Real> smom[5][MY * MX];  // (rho - 1, phi, psi, I) per cell
  __shared__ R4<Real> smu[4][UY * UX];   // (mu~rho, mu_phi, mu_psi', -) per cell

  const Geo G = a.G;
  const int tid = threadIdx.x, tx = NC * (tid % (TX / NC)), ty = tid / (TX / NC);
  const int x0 = blk.x * TX, y0 = blk.y * TY;
  const int z0 = blk.z * a.zc;
  const int z1 = min(z0 + a.zc, G.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < G.nx && y < G.ny;

  auto modn = [](int v, int n) {
    if (v < 0) v += n;
    if (v >= n) v -= n;
    if (v < 0 || v >= n) {
      v %= n;
      if (v < 0) v += n;
    }
    return v;
  };
  auto plane_src = [&](int p) { return G.wall ? min(max(p, 0), G.nz - 1) : modn(p, G.nz); };

  // asynchronous copy of ring plane p (a wall's ghost planes mirror the
  // plane next to the wall)
  auto issue_plane = [&](int p) {
    const int slot = (p + 10) % 5;
    const long long zp = (long long)plane_src(p) * G.ny;
    for (int k = tid; k < MX * MY; k += NT) {
      const int hx = k % MX, hy = k / MX;
      const int gx = modn(x0 - 2 + hx, G.nx);
      const int gy = D3 ? modn(y0 - HY + hy, G.ny) : 0;
      const long long c = (zp + gy) * G.nx + gx;
      cp_async_elem(&smom[slot][k].x, a.rho + c);
      cp_async_elem(&smom[slot][k].y, a.phi + c);
      cp_async_elem(&smom[slot][k].z, a.psi + c);
      cp_async_elem(&smom[slot][k].w, a.I + c);
    }
    cp_async_commit();
  };

  // chemical potentials of plane p on the tile plus a halo of 1
  auto compute_mu = [&](int p) {
    const int slot = (p + 8) % 4;
    if (G.wall && (p < 0 || p >= G.nz)) {  // mirror ghost: mu(-1) = mu(0), mu(nz) = mu(nz-1)
      const int src = (min(max(p, 0), G.nz - 1) + 8) % 4;
      for (int k = tid; k < UX * UY; k += NT) smu[slot][k] = smu[src][k];
      return;
    }
    const int sc = (p + 10) % 5;
    for (int k = tid; k < UX * UY; k += NT) {
      const int ux = k % UX, uy = k / UX;
      const int hx = ux + 1, hy = uy + (D3 ? 1 : 0);
      const R4<Real> cen = smom[sc][hy * MX + hx];
      Real lap[3] = {0, 0, 0};
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const R4<Real> nbv = smom[(p + L::cz(i) + 10) % 5][(hy + L::cy(i)) * MX + hx + L::cx(i)];
        const Real w = Real(L::w(i));
        lap[0] += w * (nbv.x - cen.x);
        lap[1] += w * (nbv.y - cen.y);
        lap[2] += w * (nbv.z - cen.z);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) lap[q] *= Real(6);  // 2/cs^2
      Real mr, mp, ms;
      chem_potentials<Real>(a.fe, cen.x, cen.y, cen.z, lap[0], lap[1], lap[2], cen.w, mr, mp, ms);
      smu[slot][k] = R4<Real>{mr, mp, ms, Real(0)};
    }
  };

  auto collide = [&](int zz) {
    if (!active) return;
    const int n = (zz * G.ny + y) * G.nx + x;  // the (first) cell
    // value of cell c: stored together for the two cells of a pair
    auto put = [&](auto* p, Real v0, Real v1) {
      using T = typename std::remove_pointer<decltype(p)>::type;
      if constexpr (NC == 2) store_pair(p, v0, v1);
      else *p = from_real<T>(v0);
    };
    // the cells' momenta first: their loads run under the stencil below
    Real j[NC][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if constexpr (NC == 2) {
        const auto jj = *reinterpret_cast<const R2<Real>*>(a.jm + d * G.P32 + n);
        j[0][d] = jj.x;
        j[1][d] = jj.y;
      } else {
        j[0][d] = a.jm[d * G.P32 + n];
      }
    }
    // (the cells of a pair share their brick: x is even, bricks are 4 wide)
    const bool ib = a.bflag[((zz >> 2) * a.nby + (y >> 2)) * a.nbx + (x >> 2)] != 0;
    Real drho[NC], phi[NC], psi[NC], rho[NC], F[NC][3], u[NC][3], du[NC][3], v[NC][3], us[NC][3];
    Real uu[NC], vv[NC], dus[NC], gmp[NC], gms[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int lx = tx + c;  // tile-local x of the cell
      const R4<Real> mom = smom[(zz + 10) % 5][(ty + HY) * MX + lx + 2];
      drho[c] = mom.x;
      phi[c] = mom.y;
      psi[c] = mom.z;
      rho[c] = Real(1) + drho[c];
      // gradients of the potentials (radius 1, isotropic stencil)
      Real gm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      const int ux = lx + 1, uy = ty + (D3 ? 1 : 0);
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const R4<Real> m4 = smu[(zz + L::cz(i) + 8) % 4][(uy + L::cy(i)) * UX + ux + L::cx(i)];
        const Real w = Real(L::w(i));
        const Real mv[3] = {m4.x, m4.y, m4.z};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const Real vq = w * mv[q];
          if (L::cx(i)) gm[q][0] += L::cx(i) > 0 ? vq : -vq;
          if (L::cy(i)) gm[q][1] += L::cy(i) > 0 ? vq : -vq;
          if (L::cz(i)) gm[q][2] += L::cz(i) > 0 ? vq : -vq;
        }
      }
      const R4<Real> muc = smu[(zz + 8) % 4][uy * UX + ux];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        F[c][d] = -Real(3) * (rho[c] * gm[0][d] + phi[c] * gm[1][d] + psi[c] * gm[2][d]);
        if (ib) F[c][d] += a.fib[d * G.P32 + n + c];
      }
      if (!D3) F[c][1] = 0;
      const Real irho = Real(1) / rho[c];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        u[c][d] = j[c][d] * irho;
        du[c][d] = F[c][d] * irho;
        v[c][d] = u[c][d] + Real(0.5) * du[c][d];
        us[c][d] = u[c][d] + u[c][d] + du[c][d];  // u + (u + du)
      }
      uu[c] = u[c][0] * u[c][0] + u[c][1] * u[c][1] + u[c][2] * u[c][2];
      vv[c] = v[c][0] * v[c][0] + v[c][1] * v[c][1] + v[c][2] * v[c][2];
      dus[c] = du[c][0] * us[c][0] + du[c][1] * us[c][1] + du[c][2] * us[c][2];
      gmp[c] = a.gphi * muc.y;
      gms[c] = a.gpsi * muc.z;
    }
    const int c1 = NC - 1;  // the second cell (the first again without pairs)
    if (a.mst) {
      // moment storage: the 11 values whose equilibria are this cell's
      // post-collision populations (see EqCell)
      Real* M = a.mst;
      put(M + M_DRHO * G.P32 + n, drho[0], drho[c1]);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        put(M + (M_W + d) * G.P32 + n, radd(u[0][d], du[0][d]), radd(u[c1][d], du[c1][d]));
        put(M + (M_V + d) * G.P32 + n, v[0][d], v[c1][d]);
      }
      put(M + M_PHI * G.P32 + n, phi[0], phi[c1]);
      put(M + M_GMP * G.P32 + n, gmp[0], gmp[c1]);
      put(M + M_PSI * G.P32 + n, psi[0], psi[c1]);
      put(M + M_GMS * G.P32 + n, gms[0], gms[c1]);
    } else {
      // f* = f^eq(rho, u) + w rho dP: w [drho + rho p(u)] + w rho dP; for c and
      // -c, p = A +- 3 c.u and dP = B +- 3 c.du with the shared even parts
      Real mu15[NC], md15[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        mu15[c] = rmul(Real(-1.5), uu[c]);
        md15[c] = rmul(Real(-1.5), dus[c]);
      }
      {
        const Real w0 = Real(L::w(0));
        Real f0[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c)
          f0[c] = rfma(rmul(rho[c], w0), md15[c], rmul(w0, rfma(rho[c], mu15[c], drho[c])));
        put(a.lo_dst + plane_f<L>(0) * G.P32 + n, f0[0], f0[c1]);
      }
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;
        const int o = L::opp(i);
        const Real w = Real(L::w(i));
        Real fp[NC], fm[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const Real wrho = rmul(rho[c], w);
          const Real cu = L::cx(i) * u[c][0] + L::cy(i) * u[c][1] + L::cz(i) * u[c][2];
          const Real cdu = L::cx(i) * du[c][0] + L::cy(i) * du[c][1] + L::cz(i) * du[c][2];
          const Real cus = L::cx(i) * us[c][0] + L::cy(i) * us[c][1] + L::cz(i) * us[c][2];
          const Real A = rfma(rmul(Real(4.5), cu), cu, mu15[c]);
          const Real B = rfma(rmul(Real(4.5), cdu), cus, md15[c]);
          fp[c] = rfma(wrho, rfma(Real(3), cdu, B), rmul(w, rfma(rho[c], rfma(Real(3), cu, A), drho[c])));
          fm[c] = rfma(wrho, rfma(Real(-3), cdu, B), rmul(w, rfma(rho[c], rfma(Real(-3), cu, A), drho[c])));
        }
        put(a.lo_dst + plane_f<L>(i) * G.P32 + n, fp[0], fp[c1]);
        put(a.lo_dst + plane_f<L>(o) * G.P32 + n, fm[0], fm[c1]);
      }
      // g* = g^eq(phi, mu_phi, v), h* = h^eq(psi, mu_psi', v): one velocity
      // polynomial per pair of opposite velocities serves both
      Real g3[NC], h3[NC], mv15[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        g3[c] = rmul(Real(3), gmp[c]);
        h3[c] = rmul(Real(3), gms[c]);
        mv15[c] = rmul(Real(-1.5), vv[c]);
      }
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;
        const int o = L::opp(i);
        const Real w = Real(L::w(i));
        Real gp[NC], gq[NC], hp[NC], hq[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const Real cv = L::cx(i) * v[c][0] + L::cy(i) * v[c][1] + L::cz(i) * v[c][2];
          const Real C = rfma(rmul(Real(4.5), cv), cv, mv15[c]);
          const Real pp = rfma(Real(3), cv, C), pm = rfma(Real(-3), cv, C);
          gp[c] = rmul(w, rfma(phi[c], pp, g3[c]));
          gq[c] = rmul(w, rfma(phi[c], pm, g3[c]));
          hp[c] = rmul(w, rfma(psi[c], pp, h3[c]));
          hq[c] = rmul(w, rfma(psi[c], pm, h3[c]));
        }
        put(a.lo_dst + plane_g<L>(i) * G.P32 + n, gp[0], gp[c1]);
        put(a.lo_dst + plane_g<L>(o) * G.P32 + n, gq[0], gq[c1]);
        put(a.lo_dst + plane_h<L>(i) * G.P32 + n, hp[0], hp[c1]);
        put(a.lo_dst + plane_h<L>(o) * G.P32 + n, hq[0], hq[c1]);
      }
      // rest populations close the zeroth moments: ord - 3 Gm (1 - w0) - 1.5 w0 ord v^2
      const Real w0 = Real(L::w(0));
      Real r0[NC], r1[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        r0[c] = radd(rfma(g3[c], w0 - Real(1), phi[c]), rmul(rmul(Real(-1.5) * w0, phi[c]), vv[c]));
        r1[c] = radd(rfma(h3[c], w0 - Real(1), psi[c]), rmul(rmul(Real(-1.5) * w0, psi[c]), vv[c]));
      }
      put(a.rest_dst + n, r0[0], r0[c1]);
      put(a.rest_dst + G.P32 + n, r1[0], r1[c1]);
    }
    if (ib)
#pragma unroll
      for (int d = 0; d < 3; ++d) put(a.ftot + d * G.P32 + n, F[0][d], F[c1][d]);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (!(rho[c] == rho[c]) || !(phi[c] == phi[c]) || !(psi[c] == psi[c])) atomicOr(a.status, (unsigned)ST_NAN);
  };

  // prologue: ring planes z0-2 .. z0+2; potentials z0, then z0-1 and z0+1
  // (a wall ghost copies its neighbour, so the real plane comes first); then
  // plane z0+3 into the slot of z0-2
  for (int p = z0 - 2; p <= z0 + 2; ++p) issue_plane(p);
  cp_async_wait_all();
  __syncthreads();
  compute_mu(z0);
  __syncthreads();
  compute_mu(z0 - 1);
  compute_mu(z0 + 1);
  __syncthreads();
  if (z0 + 3 <= z1 + 1) issue_plane(z0 + 3);
  cp_async_wait_all();
  __syncthreads();
  // One barrier per plane: the potentials two planes ahead are computed in
  // the same phase as the collision of this plane (their threads' uneven
  // shares of the haloed potentials even out against the collisions).
  for (int zz = z0; zz < z1; ++zz) {
    // plane zz + 4 replaces plane zz - 1 and the potentials of zz + 2 those
    // of zz - 2: neither is read in this iteration
    if (zz + 4 <= z1 + 1) issue_plane(zz + 4);
    if (zz + 2 <= z1) compute_mu(zz + 2);
    collide(zz);
    cp_async_wait_all();
    __syncthreads();
  }
}

// The collide of a form: the tau = 1 body for forms 5 and 6, else the
// general one.
template <class L, int MODE, int TX, int TY, int FORM>
__device__ __forceinline__ void collide_body(const LBArgs<MODE>& a, const Blk& blk) {
  if constexpr (form_t1<FORM>())
    collide_t1_body<L, MODE, TX, TY, FORM>(a, blk);
  else
    collide_gen_body<L, MODE, TX, TY, FORM>(a, blk);
}
// Forms of the collide: threads per SM the register budget is set for
// (0: 640; 1: 512 with the next set prefetched; 2: 768; 3: 1024; 4: 896;
// the tau = 1 collide at 5: 768 and 6: 1024).
template <int FORM> constexpr int collide_threads() {
  return FORM == 1 ? 512
                   : (FORM == 2 || FORM == 5 ? 768
                                             : (FORM == 3 || FORM == 6 ? 1024
                                                                       : (FORM == 4 ? 896 : (FORM == 8 ? 384 : (FORM == 9 ? 512 : 640)))));
}
// threads of a collide block: one per cell of the TX x TY tile, or one per
// pair of cells in the pair forms
template <int FORM, int TX, int TY> constexpr int collide_block() { return form_pair<FORM>() ? TX / 2 * TY : TX * TY; }


template <class L, int MODE, int TX, int TY, int FORM>
__global__ void __launch_bounds__(collide_block<FORM, TX, TY>(), collide_threads<FORM>() / collide_block<FORM, TX, TY>())
    k_collide(const __grid_constant__ LBArgs<MODE> a) {
  collide_body<L, MODE, TX, TY, FORM>(a, hw_blk());
}

// Calls fn(tile x, tile y, form) with the variant's compile-time values
// (3D tiles 32x4, 32x8, 64x4; 2D rows of 32, 64, 128; variant 12 is the
// smallest tile in form 4; variants 13-18 the three tiles in the tau = 1
// forms 5 and 6; variants 19-21 the three tiles of form 7, the general
// collide with the pressure-tensor force).
template <int V> using CIdx = std::integral_constant<int, V>;
template <class L, class Fn>
__host__ tlb_status collide_variant(int v, Fn&& fn) {
  constexpr bool D3 = L::DIM == 3;
  constexpr int X1 = D3 ? 32 : 64, Y1 = D3 ? 8 : 1, X2 = D3 ? 64 : 128, Y0 = D3 ? 4 : 1;
  switch (v) {
    case 1: return fn(CIdx<X1>{}, CIdx<Y1>{}, CIdx<0>{});
    case 2: return fn(CIdx<X2>{}, CIdx<Y0>{}, CIdx<0>{});
    case 3: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<1>{});
    case 4: return fn(CIdx<X1>{}, CIdx<Y1>{}, CIdx<1>{});
    case 5: return fn(CIdx<X2>{}, CIdx<Y0>{}, CIdx<1>{});
    case 6: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<2>{});
    case 7: return fn(CIdx<X1>{}, CIdx<Y1>{}, CIdx<2>{});
    case 8: return fn(CIdx<X2>{}, CIdx<Y0>{}, CIdx<2>{});
    case 9: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<3>{});
    case 10: return fn(CIdx<X1>{}, CIdx<Y1>{}, CIdx<3>{});
    case 11: return fn(CIdx<X2>{}, CIdx<Y0>{}, CIdx<3>{});
    case 12: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<4>{});  // (the larger tiles at 896 repeat 768)
    case 13: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<5>{});
    case 14: return fn(CIdx<X1>{}, CIdx<Y1>{}, CIdx<5>{});
    case 15: return fn(CIdx<X2>{}, CIdx<Y0>{}, CIdx<5>{});
    case 16: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<6>{});
    case 17: return fn(CIdx<X1>{}, CIdx<Y1>{}, CIdx<6>{});
    case 18: return fn(CIdx<X2>{}, CIdx<Y0>{}, CIdx<6>{});
    case 19: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<7>{});
    case 20: return fn(CIdx<X1>{}, CIdx<Y1>{}, CIdx<7>{});
    case 21: return fn(CIdx<X2>{}, CIdx<Y0>{}, CIdx<7>{});
    // the tau = 1 pair forms: the three tiles with 384 and 512 threads per
    // SM (two cells per thread)
    case 22: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<8>{});
    case 23: return fn(CIdx<X1>{}, CIdx<Y1>{}, CIdx<8>{});
    case 24: return fn(CIdx<X2>{}, CIdx<Y0>{}, CIdx<8>{});
    case 25: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<9>{});
    case 26: return fn(CIdx<X1>{}, CIdx<Y1>{}, CIdx<9>{});
    case 27: return fn(CIdx<X2>{}, CIdx<Y0>{}, CIdx<9>{});
    // the tau = 1 forms on 32 x 16 tiles (3D; less halo per cell): one cell
    // per thread at 768 / 1024 threads per SM, two at 384 / 512
    case 28: return fn(CIdx<32>{}, CIdx<D3 ? 16 : 1>{}, CIdx<5>{});
    case 29: return fn(CIdx<32>{}, CIdx<D3 ? 16 : 1>{}, CIdx<6>{});
    case 30: return fn(CIdx<32>{}, CIdx<D3 ? 16 : 1>{}, CIdx<8>{});
    case 31: return fn(CIdx<32>{}, CIdx<D3 ? 16 : 1>{}, CIdx<9>{});
    default: return fn(CIdx<32>{}, CIdx<Y0>{}, CIdx<0>{});
  }
}

// ------------------------------------------------------------- init & I/O
// Chemical potentials from fields in global memory (used at initialisation);
// rho holds rho - 1.
template <class L, int MODE>
__global__ void k_mu_global(Geo G, FEParams<typename Prec<MODE>::Real> fe, const typename Prec<MODE>::Real* rho,
                            const typename Prec<MODE>::Real* phi, const typename Prec<MODE>::Real* psi,
                            const typename Prec<MODE>::Real* I, typename Prec<MODE>::Real* mu) {
  using Real = typename Prec<MODE>::Real;
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= G.N) return;
  int x, y, z;
  cell_xyz(G, n, x, y, z);
  const Real* F[3] = {rho, phi, psi};
  Real lap[3] = {0, 0, 0};
  for (int i = 1; i < L::Q; ++i) {
    int sx = wrapc(x + L::cx(i), G.nx), sy = wrapc(y + L::cy(i), G.ny);
    int sz = z + L::cz(i);
    sz = G.wall ? min(max(sz, 0), G.nz - 1) : wrapc(sz, G.nz);
    long long c = ((long long)sz * G.ny + sy) * G.nx + sx;
    for (int q = 0; q < 3; ++q) lap[q] += Real(L::w(i)) * (F[q][c] - F[q][n]);
  }
  Real mr, mp, ms;
  chem_potentials<Real>(fe, rho[n], phi[n], psi[n], 6 * lap[0], 6 * lap[1], 6 * lap[2], I[n], mr, mp, ms);
  mu[n] = mr;
  mu[G.P + n] = mp;
  mu[2 * G.P + n] = ms;
}

// Equilibrium populations (eq. EDF) of the fields (rho holds rho - 1),
// stored post-collision:
// the value of direction i at cell y is the equilibrium f_i at y + c_i (or,
// across a wall, f_{opp(i)} at y), which the next pull brings back to place.
template <class L, int MODE>
__global__ void k_init_eq(Geo G, const typename Prec<MODE>::Real* rho, const typename Prec<MODE>::Real* phi,
                          const typename Prec<MODE>::Real* psi, const typename Prec<MODE>::Real* u,
                          const typename Prec<MODE>::Real* mu, typename Prec<MODE>::Real gphi,
                          typename Prec<MODE>::Real gpsi, typename Prec<MODE>::Store* lo,
                          typename Prec<MODE>::Rest* rest) {
  using Real = typename Prec<MODE>::Real;
  using Store = typename Prec<MODE>::Store;
  using Rest = typename Prec<MODE>::Rest;
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= G.N) return;
  int x, y, z;
  cell_xyz(G, n, x, y, z);
  for (int i = 0; i < L::Q; ++i) {
    int tz = z + L::cz(i);
    long long src;
    int ii = i;
    if (G.wall && (tz < 0 || tz >= G.nz)) {
      src = n;
      ii = L::opp(i);
    } else {
      src = ((long long)wrapc(tz, G.nz) * G.ny + wrapc(y + L::cy(i), G.ny)) * G.nx + wrapc(x + L::cx(i), G.nx);
    }
    Real dr = rho[src], p = phi[src], s = psi[src];
    Real r = Real(1) + dr;
    Real uv[3] = {u[src], u[G.P + src], u[2 * G.P + src]};
    Real uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
    Real cu = L::cx(ii) * uv[0] + L::cy(ii) * uv[1] + L::cz(ii) * uv[2];
    Real w = Real(L::w(ii)), w0 = Real(L::w(0));
    Real pv = eq_poly(cu, uu);
    lo[(long long)plane_f<L>(i) * G.P + n] = from_real<Store>(w * (dr + r * pv));
    Real mp = mu[G.P + src], ms = mu[2 * G.P + src];
    if (ii == 0) {
      // rest populations are stored in their own planes (direction 0 maps to itself)
      rest[n] = from_real<Rest>(p - Real(3) * gphi * mp * (Real(1) - w0) - Real(1.5) * w0 * p * uu);
      rest[G.P + n] = from_real<Rest>(s - Real(3) * gpsi * ms * (Real(1) - w0) - Real(1.5) * w0 * s * uu);
    } else {
      lo[(long long)plane_g<L>(i) * G.P + n] = from_real<Store>(w * (Real(3) * gphi * mp + p * pv));
      lo[(long long)plane_h<L>(i) * G.P + n] = from_real<Store>(w * (Real(3) * gpsi * ms + s * pv));
    }
  }
}

// Fields of the streamed populations for read-back: rho, phi, psi, u.
// Working-precision copy of a field as doubles (read-out).
template <class Real>
__global__ void k_to_double(const Real* src, long long n, double* dst) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i];
}

// Initial fields from the caller's compositions C = [3][N] (FP64 sums, then
// the working precision): rho - 1 = C1 + C2 + C3 - 1, phi = C1 - C2, psi =
// C3; or, without C, the default state: rho = 1, psi = I, phi = (1 - I)(2 s - 1)
// with the flat interface s(z) = (1 + tanh((z - z0)/(2 alpha)))/2 (s = 0
// when z0 < 0).  The velocity ([3][N], or the uniform u0) goes to uf, 2D
// fields internally as (x, 0, y).
template <class Real>
__global__ void k_init_fields(Geo G, int dim, const double* C, const double* u, double u0x, double u0y,
                              double u0z, double alpha, double z0, const Real* I, Real* rho, Real* phi,
                              Real* psi, Real* uf) {
  const long long N = G.N, P = G.P;
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  if (C) {
    rho[n] = (Real)(C[n] + C[N + n] + C[2 * N + n] - 1.0);
    phi[n] = (Real)(C[n] - C[N + n]);
    psi[n] = (Real)C[2 * N + n];
  } else {
    const long long z = n / ((long long)G.nx * G.ny);  // last axis (2D: y)
    double sv = 0.5 * (1.0 + tanh((z - z0) / (2.0 * alpha)));
    if (z0 < 0) sv = 0.0;
    const double ps = (double)I[n];
    rho[n] = (Real)0.0;
    phi[n] = (Real)((1.0 - ps) * (2.0 * sv - 1.0));
    psi[n] = (Real)ps;
  }
  const double v[3] = {u ? u[n] : u0x, u ? u[N + n] : u0y, u ? u[2 * N + n] : u0z};
  if (dim == 2) {
    uf[n] = (Real)v[0];
    uf[P + n] = 0;
    uf[2 * P + n] = (Real)v[1];
  } else {
    for (int d = 0; d < 3; ++d) uf[d * P + n] = (Real)v[d];
  }
}

template <class L, int MODE>
__global__ void k_fields(Geo G, const typename Prec<MODE>::Store* lo, const typename Prec<MODE>::Rest* rest,
                         int field, double* out /* [N], [3][N] for the velocity */) {
  using Real = typename Prec<MODE>::Real;
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= G.N) return;
  int x, y, z;
  cell_xyz(G, n, x, y, z);
  Pull<L, MODE> p;
  p.load(lo, rest, G, x, y, z);
  CellMoments<Real> m = p.moments();
  const double rho = 1.0 + (double)m.drho, phi = (double)m.phi, psi = (double)m.psi;
  switch (field) {
    case TLB_FIELD_RHO: out[n] = rho; break;
    case TLB_FIELD_PHI: out[n] = phi; break;
    case TLB_FIELD_PSI: out[n] = psi; break;
    case TLB_FIELD_C1: out[n] = 0.5 * (rho + phi - psi); break;
    case TLB_FIELD_C2: out[n] = 0.5 * (rho - phi - psi); break;
    case TLB_FIELD_C3: out[n] = psi; break;
    default:  // velocity; 2D fields are internal (x, 0, y)
      if (L::DIM == 2) {
        out[n] = (double)m.j[0] / rho;
        out[G.N + n] = (double)m.j[2] / rho;
        out[2 * G.N + n] = 0.0;
      } else {
        for (int d = 0; d < 3; ++d) out[d * G.N + n] = (double)m.j[d] / rho;
      }
  }
}

// ------------------------------------------------------------ residual
// Reference state of the equilibrium residual and the slots its maxima are
// folded into.
struct ResPtrs {
  double* snap;             // [2][P] phi, psi at the reference step
  double* xsnap;            // [nn][3] marker positions at the reference step
  unsigned long long* res;  // [3] max |change| of phi, psi, X (bit patterns)
};

// Largest change since the reference step of phi and psi (FP64 sums of the
// streamed populations) over the cells, then of the marker positions over
// the markers (virtual blocks past the cells); the reference is replaced by
// the current values.  Maxima of non-negative doubles are order independent:
// they are folded with integer atomicMax on the bit patterns, NaN mapped to
// +inf so that a diverged run never reads as converged.
template <class L, int MODE>
__device__ __forceinline__ void residual_body(const Geo& G, const typename Prec<MODE>::Store* lo,
                                              const typename Prec<MODE>::Rest* rest, const double* X, int nn,
                                              const ResPtrs& r, const Blk& blk) {
  const long long ncb = (G.N + blockDim.x - 1) / blockDim.x;
  double m[3] = {0, 0, 0};
  if (blk.x < ncb) {
    const long long n = (long long)blk.x * blockDim.x + threadIdx.x;
    if (n < G.N) {
      int x, y, z;
      cell_xyz(G, n, x, y, z);
      Pull<L, MODE> p;
      p.load(lo, rest, G, x, y, z);
      double ph = 0, ps = 0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        ph += (double)p.g[i];
        ps += (double)p.h[i];
      }
      m[0] = fabs(ph - r.snap[n]);
      m[1] = fabs(ps - r.snap[G.P + n]);
      r.snap[n] = ph;
      r.snap[G.P + n] = ps;
    }
  } else {
    const long long l = (long long)(blk.x - ncb) * blockDim.x + threadIdx.x;
    if (l < nn)
      for (int d = 0; d < 3; ++d) {
        m[2] = fmax(m[2], fabs(X[3 * l + d] - r.xsnap[3 * l + d]));
        if (!(X[3 * l + d] == X[3 * l + d])) m[2] = __longlong_as_double(0x7FF0000000000000ll);
        r.xsnap[3 * l + d] = X[3 * l + d];
      }
  }
  for (int q = 0; q < 3; ++q) {
    double v = m[q];
    if (!(v == v)) v = __longlong_as_double(0x7FF0000000000000ll);
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(r.res + q, (unsigned long long)__double_as_longlong(v));
  }
}

template <class L, int MODE>
__global__ void k_residual(Geo G, const typename Prec<MODE>::Store* lo, const typename Prec<MODE>::Rest* rest,
                           const double* X, int nn, ResPtrs r) {
  residual_body<L, MODE>(G, lo, rest, X, nn, r, hw_blk());
}

// FP64 totals: per-block partial sums of rho (as 1 + sum of deviations),
// phi and psi over a fixed cell partition, combined in fixed order by
// k_reduce_partials, so the result does not depend on scheduling.
template <class L, int MODE>
__global__ void __launch_bounds__(256) k_mass_partials(Geo G, const typename Prec<MODE>::Store* lo,
                                                       const typename Prec<MODE>::Rest* rest, double* part) {
  __shared__ double sm[3][256];
  double acc[3] = {0, 0, 0};
  for (long long n = (long long)blockIdx.x * 256 + threadIdx.x; n < G.N; n += (long long)gridDim.x * 256) {
    double r = 1.0, p = to_real(rest[n]), s = to_real(rest[G.P + n]);
    for (int i = 0; i < L::Q; ++i) r += (double)to_real(lo[(long long)plane_f<L>(i) * G.P + n]);
    for (int i = 1; i < L::Q; ++i) {
      p += (double)to_real(lo[(long long)plane_g<L>(i) * G.P + n]);
      s += (double)to_real(lo[(long long)plane_h<L>(i) * G.P + n]);
    }
    acc[0] += r;
    acc[1] += p;
    acc[2] += s;
  }
  for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[q * gridDim.x + blockIdx.x] = sm[q][0];
}

__global__ void k_reduce_partials(const double* part, int nb, int nq, double* out);
