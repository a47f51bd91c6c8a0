// FP64 CPU oracle of the ternary free-energy lattice Boltzmann + immersed
// boundary step of "Modelling ternary fluids in contact with elastic
// membranes" (Pepona, Shek, Semprebon, Krueger, Kusumaatmaja).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
// calls this file; only the tests, the smoke check and the timed CPU
// baseline of the benchmark do.  It shares no code with the CUDA path.
//
// Plain and slow on purpose: every step of the method is written in the
// order and notation of the paper, one cell at a time, in double precision.
// Where the paper is silent, the reading taken is stated at the spot.
//
// Units: lattice units, dx = dt = 1, cs^2 = 1/3 (Sec. 3.1).
// Storage: a cell (x, y, z) has index (z*ny + y)*nx + x; in 2D nz = 1 and the
// last axis is y.  Populations are stored [i][cell] for each of f, g, h.
//
// Parity status of each part (pins live in tests/test_oracle_*.py):
//   lattice, moments, equilibria, collision, streaming -- pinned (mass
//       conservation, rest-state stationarity, tau = 1 identity, Galilean
//       translation, printed D2Q9 table)
//   chemical potentials -- pinned (finite-difference variational derivative of
//       the discrete free energy; bulk minima)
//   interface physics -- pinned (tanh profile, surface tension, Laplace law)
//   membrane energies/forces -- pinned (central finite differences of the
//       energies, regular-polygon and sphere closed forms, force balance)
//   membrane profile and coupling force -- pinned (brute force on tiny inputs,
//       finite differences of the coupling energy)
//   Peskin kernel, spreading, interpolation -- pinned (moment identities,
//       exact transfer of totals and of linear fields)
//   gradient and Laplacian stencils -- pinned (analytic derivatives of
//       smooth fields, second-order convergence, mirror ghost at walls)
//   pressure-tensor force form and bulk pressure of App. A -- pinned
//       (Gibbs-Duhem relation; equal to the potential form to second order)
//   interface tensions -- pinned for all three pairs; Neumann-triangle
//       angles of a relaxed ternary lens
//   capsule area / volume -- pinned (polygon and icosahedron closed forms,
//       convergence to the sphere); contact angle -- pinned (sphere or ring
//       on a flat or tilted interface: arccos(-h/R))

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- lattice
struct Lattice {
  int Q;
  int c[19][3];
  double w[19];
  int opp[19];
};

// D2Q9 exactly as printed in Sec. 3.1 (columns of c_i; w0 = 4/9,
// w1-4 = 1/9, w5-8 = 1/36).
Lattice make_d2q9() {
  Lattice L{};
  L.Q = 9;
  const int cx[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
  for (int i = 0; i < 9; ++i) {
    L.c[i][0] = cx[i];
    L.c[i][1] = cy[i];
    L.c[i][2] = 0;
    L.w[i] = (i == 0) ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  for (int i = 0; i < 9; ++i)
    for (int k = 0; k < 9; ++k)
      if (cx[k] == -cx[i] && cy[k] == -cy[i]) L.opp[i] = k;
  return L;
}

// D3Q19: the rest velocity, the 6 face neighbours (w = 1/18) and the 12 edge
// neighbours (w = 1/36), w0 = 1/3.  The paper works in 2D and states the 3D
// extension is straightforward (Sec. 1, Sec. 5); this is the standard set.
Lattice make_d3q19() {
  Lattice L{};
  int q = 0;
  L.c[q][0] = L.c[q][1] = L.c[q][2] = 0;
  L.w[q++] = 1.0 / 3.0;
  for (int a = 0; a < 3; ++a)
    for (int s = 1; s >= -1; s -= 2) {
      L.c[q][0] = L.c[q][1] = L.c[q][2] = 0;
      L.c[q][a] = s;
      L.w[q++] = 1.0 / 18.0;
    }
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b)
      for (int sa = 1; sa >= -1; sa -= 2)
        for (int sb = 1; sb >= -1; sb -= 2) {
          L.c[q][0] = L.c[q][1] = L.c[q][2] = 0;
          L.c[q][a] = sa;
          L.c[q][b] = sb;
          L.w[q++] = 1.0 / 36.0;
        }
  L.Q = q;  // 19
  for (int i = 0; i < L.Q; ++i)
    for (int k = 0; k < L.Q; ++k)
      if (L.c[k][0] == -L.c[i][0] && L.c[k][1] == -L.c[i][1] && L.c[k][2] == -L.c[i][2])
        L.opp[i] = k;
  return L;
}

}  // namespace

extern "C" {

// Parameters, in the notation of Sec. 2.5 and Sec. 3.1.
typedef struct {
  int dim, nx, ny, nz, wall_last, pad;
  double tau, tau_phi, tau_psi, gamma_phi, gamma_psi, alpha;
  double kappa1, kappa2, kappa3, kappa_c, dc;
  double u0x, u0y, u0z, interface_pos;
  int storage;        // population storage emulated after every step:
                      // 0 none (FP64), 1 binary32, 2 binary16, 3 bfloat16
  int forcing;        // 0: exact difference method (eq. LBE); 1: Guo forcing
  int force_form;     // 0: potential form of f_FE (eq. ForceFE through eq.
                      // GradPT); 1: divergence of the explicit pressure
                      // tensor of App. A
} or_params;

}  // extern "C"

namespace {

const double CS2 = 1.0 / 3.0;

struct Membrane {
  int kind;  // 0 ring (2D), 1 triangles (3D)
  int nn, ne;
  std::vector<double> X;  // nn*3
  std::vector<int> E;     // ne*2 or ne*3
  double ks, kb, G, C;
  std::vector<double> ds0;    // 2D: initial length of segment l (node l to l+1)
  std::vector<double> A0;     // 3D: reference triangle area
  std::vector<double> G0inv;  // 3D: inverse reference metric (3 per triangle)
  std::vector<std::vector<int>> vtri;  // 3D: triangles incident to each vertex
};

struct BandCell {
  long cell;
  int mem, elem;
  double beta[3];  // barycentric weights of the closest point P
  double r[3];     // x - P (minimum image)
  double dist;     // |x - P|
  double sgn;      // +1 inside, -1 outside
  double d;        // signed distance (unclamped, |d| < dc)
};

struct Sim {
  or_params p;
  Lattice L;
  int dim;
  int n[3];
  long N;
  std::vector<double> f, g, h;  // [Q][N], populations at the start of a step
  std::vector<Membrane> mem;
  // quantities of the most recent step (kept for inspection)
  std::vector<double> rho, phi, psi, j;  // j: [3][N]
  std::vector<double> I, dsel;
  std::vector<double> mur, muphi, mupsi;
  std::vector<double> F;    // [3][N] total force used in the last collision
  std::vector<double> fib;  // [3][N]
  std::vector<BandCell> band;
  long t;
};

inline int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}
inline double wrapd(double a, double n) {  // minimum image in [-n/2, n/2)
  return a - n * std::floor(a / n + 0.5);
}
inline long cidx(const Sim& s, int x, int y, int z) {
  return ((long)z * s.n[1] + y) * s.n[0] + x;
}
inline void ccoords(const Sim& s, long c, int* x) {
  x[0] = (int)(c % s.n[0]);
  x[1] = (int)((c / s.n[0]) % s.n[1]);
  x[2] = (int)(c / ((long)s.n[0] * s.n[1]));
}
inline bool is_wall_axis(const Sim& s, int a) { return s.p.wall_last && a == s.dim - 1; }

// Neighbour for the finite-difference stencils: periodic, except across a
// wall where the mirror ghost a(-1) = a(0) is used, i.e. zero normal
// gradient, the natural boundary condition of eq. NaturalBCs.
inline long stencil_nb(const Sim& s, const int* x, const int* c) {
  int q[3];
  for (int a = 0; a < 3; ++a) {
    int v = x[a] + c[a];
    if (is_wall_axis(s, a))
      v = std::min(std::max(v, 0), s.n[a] - 1);
    else
      v = wrapi(v, s.n[a]);
    q[a] = v;
  }
  return cidx(s, q[0], q[1], q[2]);
}

// Isotropic lattice Laplacian and gradient on the velocity set of the LB
// (the paper does not print its finite-difference stencils):
//   lap a = (2/cs^2) sum_i w_i (a(x+c_i) - a(x)),  grad a = (1/cs^2) sum_i w_i c_i a(x+c_i)
double lap(const Sim& s, const std::vector<double>& a, long c) {
  int x[3];
  ccoords(s, c, x);
  double acc = 0.0;
  for (int i = 1; i < s.L.Q; ++i) acc += s.L.w[i] * (a[stencil_nb(s, x, s.L.c[i])] - a[c]);
  return 2.0 / CS2 * acc;
}
void grad(const Sim& s, const std::vector<double>& a, long c, double* gout) {
  int x[3];
  ccoords(s, c, x);
  gout[0] = gout[1] = gout[2] = 0.0;
  for (int i = 1; i < s.L.Q; ++i) {
    double v = a[stencil_nb(s, x, s.L.c[i])];
    for (int k = 0; k < 3; ++k) gout[k] += s.L.w[i] * s.L.c[i][k] * v;
  }
  for (int k = 0; k < 3; ++k) gout[k] /= CS2;
}

// ---------------------------------------------------- equilibria (eq. EDF)
inline double cdot(const Lattice& L, int i, const double* u) {
  return L.c[i][0] * u[0] + L.c[i][1] * u[1] + L.c[i][2] * u[2];
}
// f_i^eq(rho, u) = w_i rho [1 + c.u/cs^2 + uu:(cc - cs^2 I)/(2 cs^4)]
double feq(const Lattice& L, int i, double rho, const double* u) {
  double cu = cdot(L, i, u);
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return L.w[i] * rho * (1.0 + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
}
// g_i^eq / h_i^eq for i != 0: w_i [Gamma mu/cs^2 + a c.v/cs^2 + a vv:(cc - cs^2 I)/(2 cs^4)];
// the rest population closes the zeroth moment: a - sum_{i != 0}.
void oeq(const Lattice& L, double a, double Gamma, double mu, const double* v, double* out) {
  double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double sum = 0.0;
  for (int i = 1; i < L.Q; ++i) {
    double cv = cdot(L, i, v);
    out[i] = L.w[i] * (Gamma * mu / CS2 + a * cv / CS2 + a * (cv * cv - CS2 * vv) / (2.0 * CS2 * CS2));
    sum += out[i];
  }
  out[0] = a - sum;
}

// --------------------------------------------------- chemical potentials
// Appendix A, eq. AppA, with the ideal-gas part cs^2 (ln rho + 1) removed
// from mu_rho (its gradient cancels the divergence of rho cs^2 I in eq.
// ForceFE; the LB supplies that pressure itself).  mu_psi' adds the coupling
// term kappa_c (psi - I) (Sec. 2.6, below eq. EDF).
void chem_pot(const or_params& p, double rho, double phi, double psi, double Lr, double Lp,
              double Ls, double I, double* mr, double* mp, double* ms) {
  const double k1 = p.kappa1, k2 = p.kappa2, k3 = p.kappa3, a2 = p.alpha * p.alpha;
  double A = rho + phi - psi, B = rho - phi - psi;
  double tA = k1 / 8.0 * A * (A - 1.0) * (A - 2.0);
  double tB = k2 / 8.0 * B * (B - 1.0) * (B - 2.0);
  *mr = tA + tB + a2 / 4.0 * ((k1 + k2) * (Ls - Lr) + (k2 - k1) * Lp);
  *mp = tA - tB + a2 / 4.0 * ((k2 - k1) * (Lr - Ls) - (k1 + k2) * Lp);
  *ms = -tA - tB + a2 / 4.0 * ((k1 + k2) * Lr - (k2 - k1) * Lp - (k1 + k2 + 4.0 * k3) * Ls) +
        k3 * psi * (psi - 1.0) * (2.0 * psi - 1.0) + p.kappa_c * (psi - I);
}

// -------------------------------------------- Peskin kernel (eq. DiscreteDirac)
double peskin(double r) {
  double a = std::fabs(r);
  if (a <= 1.0) return (3.0 - 2.0 * a + std::sqrt(std::max(0.0, 1.0 + 4.0 * a - 4.0 * a * a))) / 8.0;
  if (a <= 2.0) return (5.0 - 2.0 * a - std::sqrt(std::max(0.0, -7.0 + 12.0 * a - 4.0 * a * a))) / 8.0;
  return 0.0;
}

// ------------------------------------------------------------ dual numbers
// Forward-mode derivatives for the 3D membrane energies (exact to round-off).
template <int W>
struct Dual {
  double v;
  double d[W];
  Dual() : v(0) { std::memset(d, 0, sizeof(d)); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof(d)); }
};
template <int W> Dual<W> operator+(const Dual<W>& a, const Dual<W>& b) { Dual<W> r; r.v = a.v + b.v; for (int k = 0; k < W; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
template <int W> Dual<W> operator-(const Dual<W>& a, const Dual<W>& b) { Dual<W> r; r.v = a.v - b.v; for (int k = 0; k < W; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
template <int W> Dual<W> operator*(const Dual<W>& a, const Dual<W>& b) { Dual<W> r; r.v = a.v * b.v; for (int k = 0; k < W; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
template <int W> Dual<W> operator/(const Dual<W>& a, const Dual<W>& b) { Dual<W> r; r.v = a.v / b.v; for (int k = 0; k < W; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v); return r; }
template <int W> Dual<W> operator*(double s, const Dual<W>& a) { Dual<W> r; r.v = s * a.v; for (int k = 0; k < W; ++k) r.d[k] = s * a.d[k]; return r; }
template <int W> Dual<W> dsqrt(const Dual<W>& a) { Dual<W> r; r.v = std::sqrt(a.v); for (int k = 0; k < W; ++k) r.d[k] = a.d[k] / (2.0 * r.v); return r; }
template <int W> struct V3 { Dual<W> x[3]; };
template <int W> V3<W> vsub(const V3<W>& a, const V3<W>& b) { V3<W> r; for (int k = 0; k < 3; ++k) r.x[k] = a.x[k] - b.x[k]; return r; }
template <int W> Dual<W> vdot(const V3<W>& a, const V3<W>& b) { return a.x[0] * b.x[0] + a.x[1] * b.x[1] + a.x[2] * b.x[2]; }
template <int W> V3<W> vcross(const V3<W>& a, const V3<W>& b) {
  V3<W> r;
  r.x[0] = a.x[1] * b.x[2] - a.x[2] * b.x[1];
  r.x[1] = a.x[2] * b.x[0] - a.x[0] * b.x[2];
  r.x[2] = a.x[0] * b.x[1] - a.x[1] * b.x[0];
  return r;
}

// ------------------------------------------------------ membrane mechanics
// 2D stretching energy, eq. DiscreteSE, with Delta s the initial length of
// each segment (the text calls it the initial marker distance).
double ring_stretch_energy(const Membrane& m, const double* X) {
  double E = 0.0;
  for (int l = 0; l < m.nn; ++l) {
    int l1 = (l + 1) % m.nn;
    double dx = X[3 * l1] - X[3 * l], dy = X[3 * l1 + 1] - X[3 * l + 1];
    double Lc = std::sqrt(dx * dx + dy * dy);
    double e = Lc / m.ds0[l] - 1.0;
    E += 0.5 * m.ks * e * e * m.ds0[l];
  }
  return E;
}
// Strain force, eq. DiscreteSF: node l receives -k_s (L_{l-1}/ds - 1) t_{l-1}
// from segment l-1 and +k_s (L_l/ds - 1) t_l from segment l.
void ring_stretch_force(const Membrane& m, const double* X, double* F) {
  for (int mm = 0; mm < m.nn; ++mm) {
    int m1 = (mm + 1) % m.nn;
    double dx = X[3 * m1] - X[3 * mm], dy = X[3 * m1 + 1] - X[3 * mm + 1];
    double Lc = std::sqrt(dx * dx + dy * dy);
    double T = m.ks * (Lc / m.ds0[mm] - 1.0);
    double tx = dx / Lc, ty = dy / Lc;
    // -dE/dX_{m+1} = -T t ; -dE/dX_m = +T t
    F[3 * m1] -= T * tx;
    F[3 * m1 + 1] -= T * ty;
    F[3 * mm] += T * tx;
    F[3 * mm + 1] += T * ty;
  }
}
// 2D bending energy, eq. DiscreteBE with eq. DiscreteTheta (Delta theta =
// 2 arccos y, taken literally) and eq. DiscreteArcLength.
double ring_bend_energy(const Membrane& m, const double* X) {
  double E = 0.0;
  for (int l = 0; l < m.nn; ++l) {
    int lp = (l + 1) % m.nn, lm = (l + m.nn - 1) % m.nn;
    double ax = X[3 * lp] - X[3 * l], ay = X[3 * lp + 1] - X[3 * l + 1];
    double bx = X[3 * l] - X[3 * lm], by = X[3 * l + 1] - X[3 * lm + 1];
    double la = std::sqrt(ax * ax + ay * ay), lb = std::sqrt(bx * bx + by * by);
    double y = (ax * bx + ay * by) / (la * lb);
    y = std::min(1.0, std::max(-1.0, y));
    double dth = 2.0 * std::acos(y);
    E += 0.25 * m.kb * dth * dth / (la + lb);
  }
  return E;
}
// Bending force, eq. DiscreteBF.  The factor 2 dtheta * d(dtheta)/dy equals
// -8 theta1 / sin(theta1) with theta1 = arccos y; it is evaluated through
// that ratio (series 1 + theta1^2/6 for theta1 < 1e-4), which keeps the
// straight configuration y -> 1 finite.
void ring_bend_force(const Membrane& m, const double* X, double* F) {
  for (int mm = 0; mm < m.nn; ++mm) {
    int mp = (mm + 1) % m.nn, mq = (mm + m.nn - 1) % m.nn;
    double a[2] = {X[3 * mp] - X[3 * mm], X[3 * mp + 1] - X[3 * mm + 1]};
    double b[2] = {X[3 * mm] - X[3 * mq], X[3 * mm + 1] - X[3 * mq + 1]};
    double la = std::sqrt(a[0] * a[0] + a[1] * a[1]), lb = std::sqrt(b[0] * b[0] + b[1] * b[1]);
    double ab = a[0] * b[0] + a[1] * b[1];
    double y = std::min(1.0, std::max(-1.0, ab / (la * lb)));
    double th1 = std::acos(y);
    double ratio = th1 < 1e-4 ? 1.0 + th1 * th1 / 6.0 : th1 / std::sin(th1);
    double dth = 2.0 * th1, dsp = la + lb;
    double cE = 0.25 * m.kb;
    // dy/da, dy/db
    double dya[2], dyb[2];
    for (int k = 0; k < 2; ++k) {
      dya[k] = b[k] / (la * lb) - ab * a[k] / (la * la * la * lb);
      dyb[k] = a[k] / (la * lb) - ab * b[k] / (la * lb * lb * lb);
    }
    // dE_m/dX = cE [ (-8 ratio / dsp) dy/dX - (dth/dsp)^2 d(dsp)/dX ]
    double k1 = cE * (-8.0 * ratio / dsp);
    double k2 = cE * (dth / dsp) * (dth / dsp);
    double ua[2] = {a[0] / la, a[1] / la}, ub[2] = {b[0] / lb, b[1] / lb};
    for (int k = 0; k < 2; ++k) {
      // a = X_{m+1} - X_m ; b = X_m - X_{m-1}
      double gp = k1 * dya[k] - k2 * ua[k];                       // d/dX_{m+1}
      double gm = k1 * (-dya[k] + dyb[k]) - k2 * (-ua[k] + ub[k]);  // d/dX_m
      double gq = k1 * (-dyb[k]) - k2 * (-ub[k]);                 // d/dX_{m-1}
      F[3 * mp + k] -= gp;
      F[3 * mm + k] -= gm;
      F[3 * mq + k] -= gq;
    }
  }
}

// 3D Skalak law per triangle (shear modulus G, area ratio C): with the
// in-plane right Cauchy-Green tensor C^ = G0^{-1} g (g, G0 the current and
// reference edge metrics), I1 = tr C^ - 2, I2 = det C^ - 1 and
// W = (G/4)(I1^2 + 2 I1 - 2 I2 + C I2^2), E_T = A0_T W.  Not in the paper
// (Sec. 1 names the Skalak law as an alternative); standard definition.
template <int W>
Dual<W> skalak_tri(const Membrane& m, int t, const V3<W>& a, const V3<W>& b, const V3<W>& c) {
  V3<W> e1 = vsub(b, a), e2 = vsub(c, a);
  Dual<W> g11 = vdot(e1, e1), g12 = vdot(e1, e2), g22 = vdot(e2, e2);
  const double* Gi = &m.G0inv[3 * t];
  Dual<W> tr = Gi[0] * g11 + 2.0 * (Gi[1] * g12) + Gi[2] * g22;
  double detG0inv = Gi[0] * Gi[2] - Gi[1] * Gi[1];
  Dual<W> det = detG0inv * (g11 * g22 - g12 * g12);
  Dual<W> I1 = tr - Dual<W>(2.0), I2 = det - Dual<W>(1.0);
  Dual<W> w = (m.G / 4.0) * (I1 * I1 + 2.0 * I1 - 2.0 * I2 + m.C * (I2 * I2));
  return m.A0[t] * w;
}

double skalak_energy(const Membrane& m, const double* X) {
  double E = 0.0;
  for (int t = 0; t < m.ne; ++t) {
    V3<1> v[3];
    for (int q = 0; q < 3; ++q)
      for (int k = 0; k < 3; ++k) v[q].x[k] = Dual<1>(X[3 * m.E[3 * t + q] + k]);
    E += skalak_tri<1>(m, t, v[0], v[1], v[2]).v;
  }
  return E;
}
void skalak_force(const Membrane& m, const double* X, double* F) {
  for (int t = 0; t < m.ne; ++t) {
    V3<9> v[3];
    for (int q = 0; q < 3; ++q)
      for (int k = 0; k < 3; ++k) {
        v[q].x[k] = Dual<9>(X[3 * m.E[3 * t + q] + k]);
        v[q].x[k].d[3 * q + k] = 1.0;
      }
    Dual<9> e = skalak_tri<9>(m, t, v[0], v[1], v[2]);
    for (int q = 0; q < 3; ++q)
      for (int k = 0; k < 3; ++k) F[3 * m.E[3 * t + q] + k] -= e.d[3 * q + k];
  }
}

// 3D Helfrich bending without spontaneous curvature (as Sec. 2.3 in 2D):
// E = (kb/2) sum_v A_v (2 H_v)^2 with the cotangent mean-curvature normal
// K_v = (1/(2 A_v)) sum_j (cot a_vj + cot b_vj)(x_v - x_j) = 2 H_v n_v and the
// mixed Voronoi area A_v of Meyer, Desbrun, Schroeder and Barr (2003), so
// E_v = kb |sum_j (...)|^2 / (8 A_v).
const int HW = 27;  // dual width: up to 9 distinct vertices around v
template <int W>
Dual<W> helfrich_vertex(const Membrane& m, int v, const std::vector<int>& loc,
                        const std::vector<V3<W>>& P) {
  // loc maps mesh vertex -> local slot in P (-1 if absent)
  V3<W> K;
  Dual<W> A(0.0);
  const V3<W>& xv = P[loc[v]];
  for (int t : m.vtri[v]) {
    int q0 = m.E[3 * t], q1 = m.E[3 * t + 1], q2 = m.E[3 * t + 2];
    int j, k;
    if (q0 == v) { j = q1; k = q2; }
    else if (q1 == v) { j = q2; k = q0; }
    else { j = q0; k = q1; }
    const V3<W>& xj = P[loc[j]];
    const V3<W>& xk = P[loc[k]];
    V3<W> vj = vsub(xv, xj), vk = vsub(xv, xk);
    // angle at j between (xv - xj) and (xk - xj); angle at k likewise
    V3<W> kj = vsub(xk, xj), jk = vsub(xj, xk);
    Dual<W> cotj = vdot(vj, kj) / dsqrt(vdot(vcross(vj, kj), vcross(vj, kj)));
    Dual<W> cotk = vdot(vk, jk) / dsqrt(vdot(vcross(vk, jk), vcross(vk, jk)));
    for (int c = 0; c < 3; ++c) K.x[c] = K.x[c] + cotk * vj.x[c] + cotj * vk.x[c];
    V3<W> ej = vsub(xj, xv), ek = vsub(xk, xv);
    Dual<W> area = 0.5 * dsqrt(vdot(vcross(ej, ek), vcross(ej, ek)));
    double dv = vdot(ej, ek).v, dj = vdot(vj, kj).v, dk = vdot(vk, jk).v;
    if (dv < 0.0)
      A = A + 0.5 * area;
    else if (dj < 0.0 || dk < 0.0)
      A = A + 0.25 * area;
    else
      A = A + 0.125 * (vdot(vj, vj) * cotk + vdot(vk, vk) * cotj);
  }
  Dual<W> K2 = vdot(K, K);
  return (m.kb / 8.0) * (K2 / A);
}

void helfrich_eval(const Membrane& m, const double* X, double* E, double* F) {
  double Et = 0.0;
  std::vector<int> loc(m.nn, -1);
  for (int v = 0; v < m.nn; ++v) {
    std::vector<int> verts;
    verts.push_back(v);
    for (int t : m.vtri[v])
      for (int q = 0; q < 3; ++q) {
        int u = m.E[3 * t + q];
        if (std::find(verts.begin(), verts.end(), u) == verts.end()) verts.push_back(u);
      }
    if ((int)verts.size() * 3 > HW) { std::fprintf(stderr, "oracle: valence too high\n"); continue; }
    std::vector<V3<HW>> P(verts.size());
    for (size_t s = 0; s < verts.size(); ++s) {
      loc[verts[s]] = (int)s;
      for (int k = 0; k < 3; ++k) {
        P[s].x[k] = Dual<HW>(X[3 * verts[s] + k]);
        if (F) P[s].x[k].d[3 * s + k] = 1.0;
      }
    }
    Dual<HW> e = helfrich_vertex<HW>(m, v, loc, P);
    Et += e.v;
    if (F)
      for (size_t s = 0; s < verts.size(); ++s)
        for (int k = 0; k < 3; ++k) F[3 * verts[s] + k] -= e.d[3 * s + k];
    for (int u : verts) loc[u] = -1;
  }
  if (E) *E = Et;
}

void membrane_setup(Membrane& m) {
  if (m.kind == 0) {
    m.ds0.resize(m.nn);
    for (int l = 0; l < m.nn; ++l) {
      int l1 = (l + 1) % m.nn;
      double dx = m.X[3 * l1] - m.X[3 * l], dy = m.X[3 * l1 + 1] - m.X[3 * l + 1];
      m.ds0[l] = std::sqrt(dx * dx + dy * dy);
    }
    m.ne = m.nn;
    m.E.resize(2 * m.nn);
    for (int l = 0; l < m.nn; ++l) { m.E[2 * l] = l; m.E[2 * l + 1] = (l + 1) % m.nn; }
  } else {
    m.A0.resize(m.ne);
    m.G0inv.resize(3 * m.ne);
    m.vtri.assign(m.nn, {});
    for (int t = 0; t < m.ne; ++t) {
      const double* a = &m.X[3 * m.E[3 * t]];
      const double* b = &m.X[3 * m.E[3 * t + 1]];
      const double* c = &m.X[3 * m.E[3 * t + 2]];
      double e1[3], e2[3];
      for (int k = 0; k < 3; ++k) { e1[k] = b[k] - a[k]; e2[k] = c[k] - a[k]; }
      double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
      double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
      double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
      double det = g11 * g22 - g12 * g12;
      m.A0[t] = 0.5 * std::sqrt(det);
      m.G0inv[3 * t] = g22 / det;
      m.G0inv[3 * t + 1] = -g12 / det;
      m.G0inv[3 * t + 2] = g11 / det;
      for (int q = 0; q < 3; ++q) m.vtri[m.E[3 * t + q]].push_back(t);
    }
  }
}

// Elastic forces F_s + F_b (eq. MembraneForces without the coupling part).
void elastic_force(const Membrane& m, const double* X, double* F) {
  if (m.kind == 0) {
    ring_stretch_force(m, X, F);
    ring_bend_force(m, X, F);
  } else {
    skalak_force(m, X, F);
    helfrich_eval(m, X, nullptr, F);
  }
}

// ----------------------------------------------------- geometry for I(x)
// Closest point of p on segment [a, b] (all relative to the cell).
void closest_seg(const double* a, const double* b, double* beta, double* P) {
  double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double l2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
  double t = l2 > 0 ? -(a[0] * ab[0] + a[1] * ab[1] + a[2] * ab[2]) / l2 : 0.0;
  t = std::min(1.0, std::max(0.0, t));
  beta[0] = 1.0 - t;
  beta[1] = t;
  beta[2] = 0.0;
  for (int k = 0; k < 3; ++k) P[k] = a[k] + t * ab[k];
}
double n3(const double* v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

// Closest point of the origin on triangle (a, b, c): the projection on the
// plane if it falls inside, else the best of the three edge projections.
void closest_tri(const double* a, const double* b, const double* c, double* beta, double* P) {
  double e1[3], e2[3];
  for (int k = 0; k < 3; ++k) { e1[k] = b[k] - a[k]; e2[k] = c[k] - a[k]; }
  double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
  double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
  double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
  double r1 = -(a[0] * e1[0] + a[1] * e1[1] + a[2] * e1[2]);
  double r2 = -(a[0] * e2[0] + a[1] * e2[1] + a[2] * e2[2]);
  double det = g11 * g22 - g12 * g12;
  double s = (g22 * r1 - g12 * r2) / det, t = (g11 * r2 - g12 * r1) / det;
  if (s >= 0 && t >= 0 && s + t <= 1) {
    beta[0] = 1 - s - t;
    beta[1] = s;
    beta[2] = t;
    for (int k = 0; k < 3; ++k) P[k] = a[k] + s * e1[k] + t * e2[k];
    return;
  }
  const double* V[3] = {a, b, c};
  double best = 1e300;
  for (int q = 0; q < 3; ++q) {
    double bb[3], PP[3];
    closest_seg(V[q], V[(q + 1) % 3], bb, PP);
    double d = n3(PP);
    if (d < best) {
      best = d;
      beta[0] = beta[1] = beta[2] = 0.0;
      beta[q] = bb[0];
      beta[(q + 1) % 3] = bb[1];
      for (int k = 0; k < 3; ++k) P[k] = PP[k];
    }
  }
}

// Inside tests (sign of d in eq. Iprofile: positive inside the capsule).
// 2D: winding number of the ring around the cell; 3D: generalized winding
// number, sum of the triangles' signed solid angles (Van Oosterom and
// Strackee 1983) over 4 pi.
double winding2d(const std::vector<double>& R, int nn) {
  double w = 0.0;
  for (int l = 0; l < nn; ++l) {
    int l1 = (l + 1) % nn;
    const double* a = &R[3 * l];
    const double* b = &R[3 * l1];
    w += std::atan2(a[0] * b[1] - a[1] * b[0], a[0] * b[0] + a[1] * b[1]);
  }
  return w / (2.0 * M_PI);
}
double winding3d(const Membrane& m, const std::vector<double>& R) {
  double w = 0.0;
  for (int t = 0; t < m.ne; ++t) {
    const double* a = &R[3 * m.E[3 * t]];
    const double* b = &R[3 * m.E[3 * t + 1]];
    const double* c = &R[3 * m.E[3 * t + 2]];
    double la = n3(a), lb = n3(b), lc = n3(c);
    double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    double det = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
    double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    double bcd = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
    double ca = c[0] * a[0] + c[1] * a[1] + c[2] * a[2];
    double den = la * lb * lc + ab * lc + bcd * la + ca * lb;
    w += 2.0 * std::atan2(det, den);
  }
  return w / (4.0 * M_PI);
}

// Contiguous copy of a membrane on a periodic lattice: markers are unwrapped
// along the mesh edges (every edge is shorter than half the domain), so the
// copy is one connected closed curve / surface.
struct Contig {
  std::vector<double> X;
  double lo[3], hi[3];
};
Contig make_contig(const Sim& s, const Membrane& m, const double* X) {
  Contig c;
  c.X.assign(3 * m.nn, 0.0);
  std::vector<char> done(m.nn, 0);
  std::vector<std::vector<int>> nb(m.nn);
  int nv = (m.kind == 0) ? 2 : 3;
  for (int e = 0; e < m.ne; ++e)
    for (int q = 0; q < nv; ++q) {
      int a = m.E[nv * e + q], b = m.E[nv * e + (q + 1) % nv];
      nb[a].push_back(b);
      nb[b].push_back(a);
    }
  for (int r0 = 0; r0 < m.nn; ++r0) {
    if (done[r0]) continue;
    for (int k = 0; k < 3; ++k) c.X[3 * r0 + k] = X[3 * r0 + k];
    done[r0] = 1;
    std::vector<int> stack{r0};
    while (!stack.empty()) {
      int a = stack.back();
      stack.pop_back();
      for (int b : nb[a]) {
        if (done[b]) continue;
        for (int k = 0; k < 3; ++k) {
          double r = X[3 * b + k] - X[3 * a + k];
          if (k < s.dim && !is_wall_axis(s, k)) r = wrapd(r, s.n[k]);
          c.X[3 * b + k] = c.X[3 * a + k] + r;
        }
        done[b] = 1;
        stack.push_back(b);
      }
    }
  }
  for (int k = 0; k < 3; ++k) { c.lo[k] = 1e300; c.hi[k] = -1e300; }
  for (int l = 0; l < m.nn; ++l)
    for (int k = 0; k < 3; ++k) {
      c.lo[k] = std::min(c.lo[k], c.X[3 * l + k]);
      c.hi[k] = std::max(c.hi[k], c.X[3 * l + k]);
    }
  return c;
}

// Signed distance of one cell to one membrane (eq. Iprofile): nearest
// segment / triangle over the periodic images of the membrane (lowest
// element index, then lowest image, on ties), sign from the winding number
// (inside any image).  Reading: the paper does not say how d is discretised;
// the distance to the polyline / triangulated surface avoids the ripple that
// marker-to-cell distances would give.  Images farther than dc + 1 from the
// cell (bounding-box test) are skipped: they are clamped anyway and add no
// winding.  Returns false when every image is that far.
bool cell_distance(const Sim& s, const Membrane& m, const Contig& cg, const int* xc,
                   BandCell* out) {
  const double dc = s.p.dc;
  int per[3] = {0, 0, 0};
  for (int k = 0; k < s.dim; ++k) per[k] = is_wall_axis(s, k) ? 0 : 1;
  bool any = false;
  double best = 1e300, wsum = 0.0;
  unsigned long long bestk = 0;
  int be = -1;
  double bb[3] = {0, 0, 0}, bP[3] = {0, 0, 0};
  std::vector<double> R(3 * m.nn);
  for (int i0 = -per[0]; i0 <= per[0]; ++i0)
    for (int i1 = -per[1]; i1 <= per[1]; ++i1)
      for (int i2 = -per[2]; i2 <= per[2]; ++i2) {
        double sh[3] = {(double)i0 * s.n[0], (double)i1 * s.n[1], (double)i2 * s.n[2]};
        double gap2 = 0.0;
        for (int k = 0; k < s.dim; ++k) {
          double lo = cg.lo[k] + sh[k] - xc[k], hi = cg.hi[k] + sh[k] - xc[k];
          double g = std::max(0.0, std::max(lo, -hi));
          gap2 += g * g;
        }
        if (gap2 > (dc + 1.0) * (dc + 1.0)) continue;
        any = true;
        for (int l = 0; l < m.nn; ++l)
          for (int k = 0; k < 3; ++k)
            R[3 * l + k] = (k < s.dim) ? cg.X[3 * l + k] + sh[k] - xc[k] : 0.0;
        for (int e = 0; e < m.ne; ++e) {
          double beta[3], P[3];
          if (m.kind == 0)
            closest_seg(&R[3 * m.E[2 * e]], &R[3 * m.E[2 * e + 1]], beta, P);
          else
            closest_tri(&R[3 * m.E[3 * e]], &R[3 * m.E[3 * e + 1]], &R[3 * m.E[3 * e + 2]], beta, P);
          double d = n3(P);
          // nearest element, distances compared on a grid of 2^-34 lattice
          // units and ties broken by the lowest element index (reading: the
          // paper leaves ties open; exact mirror-symmetric ties would
          // otherwise be decided by rounding)
          unsigned long long kd = (unsigned long long)(d * 17179869184.0);
          if (be < 0 || kd < bestk) {
            bestk = kd;
            best = d;
            be = e;
            std::memcpy(bb, beta, sizeof(bb));
            std::memcpy(bP, P, sizeof(bP));
          }
        }
        wsum += (m.kind == 0) ? winding2d(R, m.nn) : winding3d(m, R);
      }
  if (!any) return false;
  out->elem = be;
  std::memcpy(out->beta, bb, sizeof(bb));
  for (int k = 0; k < 3; ++k) out->r[k] = -bP[k];  // x - P
  out->dist = best;
  out->sgn = (std::fabs(wsum) > 0.5) ? 1.0 : -1.0;
  out->d = out->sgn * best;
  return true;
}

// Membrane profile I (eq. Iprofile) for all cells, with d clamped to
// [-dc, dc] and, for several capsules, the largest signed distance.  Cells
// with |d| < dc form the band that feels the coupling force.
void iprofile(const Sim& s, const std::vector<const double*>& Xs, std::vector<double>& I,
              std::vector<double>& dsel, std::vector<BandCell>& band) {
  const double dc = s.p.dc, al = s.p.alpha;
  I.assign(s.N, 0.0);
  dsel.assign(s.N, 0.0);
  std::vector<BandCell> cb(s.N);
  std::vector<char> inb(s.N, 0);
  std::vector<Contig> cgs;
  for (size_t mi = 0; mi < s.mem.size(); ++mi) cgs.push_back(make_contig(s, s.mem[mi], Xs[mi]));
#pragma omp parallel for schedule(dynamic, 64)
  for (long c = 0; c < s.N; ++c) {
    int xc[3];
    ccoords(s, c, xc);
    double bestd = -1e300;
    BandCell bestc{};
    bool have = false;
    for (size_t mi = 0; mi < s.mem.size(); ++mi) {
      BandCell bc{};
      double dm = -dc;
      if (cell_distance(s, s.mem[mi], cgs[mi], xc, &bc)) dm = std::min(dc, std::max(-dc, bc.d));
      if (dm > bestd) {
        bestd = dm;
        have = std::fabs(dm) < dc && bc.elem >= 0;
        bc.mem = (int)mi;
        bc.cell = c;
        bestc = bc;
      }
    }
    if (s.mem.empty()) bestd = -dc;
    dsel[c] = bestd;
    I[c] = 0.5 * (1.0 + std::tanh(bestd / (2.0 * al)));
    if (have) { cb[c] = bestc; inb[c] = 1; }
  }
  band.clear();
  for (long c = 0; c < s.N; ++c)
    if (inb[c]) band.push_back(cb[c]);
}

// Coupling force on the markers, eq. DiscreteCF derived from eq.
// DiscreteCE: F_c,k = sum_x kappa_c (psi - I) dI/dd dd/dX_k with
// dI/dd = sech^2(d/(2 alpha))/(4 alpha) and, for closest point
// P = sum_k beta_k X_k, dd/dX_k = -sgn beta_k (x - P)/|x - P|.  Reading: the
// sign follows from differentiating the energy (the printed formula carries
// an extra minus).  At |x - P| ~ 0 the outward element normal is used.
void coupling_force(const Sim& s, const std::vector<const double*>& Xs, const std::vector<BandCell>& band,
                    const std::vector<double>& psi, const std::vector<double>& I,
                    std::vector<std::vector<double>>& F) {
  const double al = s.p.alpha;
  for (const BandCell& b : band) {
    const Membrane& m = s.mem[b.mem];
    const double* X = Xs[b.mem];
    double ch = std::cosh(b.d / (2.0 * al));
    double coef = s.p.kappa_c * (psi[b.cell] - I[b.cell]) / (ch * ch) / (4.0 * al);
    double dir[3];
    if (b.dist > 1e-12) {
      for (int k = 0; k < 3; ++k) dir[k] = -b.sgn * b.r[k] / b.dist;
    } else {
      double nrm[3] = {0, 0, 0};
      if (m.kind == 0) {
        int a = m.E[2 * b.elem], c2 = m.E[2 * b.elem + 1];
        double tx = X[3 * c2] - X[3 * a], ty = X[3 * c2 + 1] - X[3 * a + 1];
        double l = std::sqrt(tx * tx + ty * ty);
        nrm[0] = ty / l;
        nrm[1] = -tx / l;
      } else {
        const double* a = &X[3 * m.E[3 * b.elem]];
        const double* bb = &X[3 * m.E[3 * b.elem + 1]];
        const double* cc = &X[3 * m.E[3 * b.elem + 2]];
        double e1[3] = {bb[0] - a[0], bb[1] - a[1], bb[2] - a[2]};
        double e2[3] = {cc[0] - a[0], cc[1] - a[1], cc[2] - a[2]};
        nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double l = n3(nrm);
        for (int k = 0; k < 3; ++k) nrm[k] /= l;
      }
      for (int k = 0; k < 3; ++k) dir[k] = nrm[k];
    }
    int nv = (m.kind == 0) ? 2 : 3;
    for (int q = 0; q < nv; ++q) {
      int node = m.E[nv * b.elem + q];
      for (int k = 0; k < s.dim; ++k) F[b.mem][3 * node + k] += coef * b.beta[q] * dir[k];
    }
  }
}

// Spreading, eq. Spreading with eq. DiscreteDirac: f_IB(x) = sum_l F_l
// delta_h(x - X_l).  Reading: F_l = -dE/dX_l is already a nodal force, so
// the arc-length factor Delta s is taken as 1 (it equals dx = 1 by
// construction of the markers, Sec. 3.2).
void spread(const Sim& s, const std::vector<const double*>& Xs,
            const std::vector<std::vector<double>>& F, std::vector<double>& fib) {
  fib.assign(3 * s.N, 0.0);
  for (size_t mi = 0; mi < s.mem.size(); ++mi) {
    const Membrane& m = s.mem[mi];
    for (int l = 0; l < m.nn; ++l) {
      const double* Xl = &Xs[mi][3 * l];
      int base[3] = {0, 0, 0}, span[3] = {1, 1, 1};
      for (int k = 0; k < s.dim; ++k) { base[k] = (int)std::floor(Xl[k]) - 1; span[k] = 4; }
      for (int a = 0; a < span[0]; ++a)
        for (int b = 0; b < span[1]; ++b)
          for (int c = 0; c < span[2]; ++c) {
            int q[3] = {base[0] + a, base[1] + b, base[2] + c};
            double wgt = 1.0;
            for (int k = 0; k < s.dim; ++k) wgt *= peskin(q[k] - Xl[k]);
            if (wgt == 0.0) continue;
            bool out = false;
            for (int k = 0; k < 3; ++k) {
              if (is_wall_axis(s, k)) { if (q[k] < 0 || q[k] >= s.n[k]) out = true; }
              else q[k] = wrapi(q[k], s.n[k]);
            }
            if (out) continue;
            long cc = cidx(s, q[0], q[1], q[2]);
            for (int k = 0; k < s.dim; ++k) fib[3 * cc + k] += wgt * F[mi][3 * l + k];
          }
    }
  }
}

// Interpolation, eq. Interpolation: U_l = sum_x v(x) delta_h(x - X_l).
void interp(const Sim& s, const double* X, int nn, const std::vector<double>& v, double* U) {
  for (int l = 0; l < nn; ++l) {
    const double* Xl = &X[3 * l];
    int base[3] = {0, 0, 0}, span[3] = {1, 1, 1};
    for (int k = 0; k < s.dim; ++k) { base[k] = (int)std::floor(Xl[k]) - 1; span[k] = 4; }
    double u[3] = {0, 0, 0};
    for (int a = 0; a < span[0]; ++a)
      for (int b = 0; b < span[1]; ++b)
        for (int c = 0; c < span[2]; ++c) {
          int q[3] = {base[0] + a, base[1] + b, base[2] + c};
          double wgt = 1.0;
          for (int k = 0; k < s.dim; ++k) wgt *= peskin(q[k] - Xl[k]);
          if (wgt == 0.0) continue;
          bool out = false;
          for (int k = 0; k < 3; ++k) {
            if (is_wall_axis(s, k)) { if (q[k] < 0 || q[k] >= s.n[k]) out = true; }
            else q[k] = wrapi(q[k], s.n[k]);
          }
          if (out) continue;
          long cc = cidx(s, q[0], q[1], q[2]);
          for (int k = 0; k < s.dim; ++k) u[k] += wgt * v[3 * cc + k];
        }
    for (int k = 0; k < 3; ++k) U[3 * l + k] = u[k];
  }
}

// ------------------------------------------------- storage rounding
// Round x to the nearest number with `p` significant bits (ties to even),
// subnormals below 2^emin on the fixed grid of spacing 2^(emin - p + 1),
// overflow past the largest finite value to infinity: the IEEE 754
// binary16 (p = 11, emin = -14, max 65504), bfloat16 (p = 8, emin = -126)
// and binary32 (p = 24, emin = -126) formats written from their definition.
double round_to_format(double x, int p, int emin, double maxv) {
  if (x == 0.0 || !std::isfinite(x)) return x;
  int e;
  std::frexp(x, &e);  // |x| = m 2^e, m in [0.5, 1)
  int ex = e - 1;     // |x| in [2^ex, 2^(ex+1))
  if (ex < emin) ex = emin;
  double q = std::ldexp(1.0, ex - (p - 1));     // spacing of the grid at |x|
  double r = std::nearbyint(x / q) * q;          // default rounding: ties to even
  if (std::fabs(r) > maxv) return x > 0 ? INFINITY : -INFINITY;
  return r;
}

// Storage emulation: the stored quantities are f_i - w_i, g_i and h_i for
// i != 0 in the storage format, and g_0, h_0 (they carry phi and psi) in
// binary32 when the storage format is 16 bits wide.
void emulate_storage(Sim& s) {
  const int st = s.p.storage;
  if (st == 0) return;
  int p = 24, emin = -126;
  double maxv = 3.4028234663852886e38;
  if (st == 2) { p = 11; emin = -14; maxv = 65504.0; }
  if (st == 3) { p = 8; emin = -126; maxv = 3.3895313892515355e38; }
  const int Q = s.L.Q;
  const long N = s.N;
#pragma omp parallel for
  for (long c = 0; c < N; ++c)
    for (int i = 0; i < Q; ++i) {
      long k = (long)i * N + c;
      s.f[k] = round_to_format(s.f[k] - s.L.w[i], p, emin, maxv) + s.L.w[i];
      if (i == 0) {
        s.g[k] = round_to_format(s.g[k], 24, -126, 3.4028234663852886e38);
        s.h[k] = round_to_format(s.h[k], 24, -126, 3.4028234663852886e38);
      } else {
        s.g[k] = round_to_format(s.g[k], p, emin, maxv);
        s.h[k] = round_to_format(s.h[k], p, emin, maxv);
      }
    }
}

// ------------------------------------------------------------ the step
void moments(Sim& s) {
  const int Q = s.L.Q;
  s.rho.assign(s.N, 0.0);
  s.phi.assign(s.N, 0.0);
  s.psi.assign(s.N, 0.0);
  s.j.assign(3 * s.N, 0.0);
#pragma omp parallel for
  for (long c = 0; c < s.N; ++c) {
    double r = 0, ph = 0, ps = 0, jj[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      double fi = s.f[(long)i * s.N + c];
      r += fi;
      for (int k = 0; k < 3; ++k) jj[k] += s.L.c[i][k] * fi;
      ph += s.g[(long)i * s.N + c];
      ps += s.h[(long)i * s.N + c];
    }
    s.rho[c] = r;
    s.phi[c] = ph;
    s.psi[c] = ps;
    for (int k = 0; k < 3; ++k) s.j[3 * c + k] = jj[k];
  }
}

void potentials(Sim& s) {
  s.mur.assign(s.N, 0.0);
  s.muphi.assign(s.N, 0.0);
  s.mupsi.assign(s.N, 0.0);
#pragma omp parallel for
  for (long c = 0; c < s.N; ++c)
    chem_pot(s.p, s.rho[c], s.phi[c], s.psi[c], lap(s, s.rho, c), lap(s, s.phi, c),
             lap(s, s.psi, c), s.I[c], &s.mur[c], &s.muphi[c], &s.mupsi[c]);
}

// Bulk pressure p_b of App. A (the ideal-gas part rho cs^2 included).
// Reading: the printed polynomial does not satisfy the Gibbs-Duhem relation
// grad p_b = rho grad mu_rho^b + phi grad mu_phi^b + psi grad mu_psi^b of the
// bulk free energy of eq. LandauFE; it is short by 3 (kappa_1 + kappa_2)
// psi^2 / 32, which is not a constant.  That term is added here (the last
// line), so that p_b = rho cs^2 + sum_m C_m dF/dC_m - F_b exactly.
double bulk_pressure(const or_params& p, double r, double f, double s) {
  const double k1 = p.kappa1, k2 = p.kappa2, k3 = p.kappa3;
  const double r2 = r * r, f2 = f * f, s2 = s * s;
  double pb = r * CS2;
  pb += (k1 + k2) * (3.0 / 32 * r2 * r2 + 3.0 / 32 * f2 * f2 + 9.0 / 16 * r2 * f2 + 9.0 / 16 * r2 * s2 +
                     9.0 / 16 * f2 * s2 - 3.0 / 8 * r2 * r * s - 3.0 / 8 * r * s2 * s + 3.0 / 4 * r2 * s -
                     3.0 / 4 * r * f2 - 3.0 / 4 * r * s2 + 3.0 / 4 * f2 * s - 1.0 / 4 * r2 * r + 1.0 / 8 * r2 +
                     1.0 / 8 * f2 - 1.0 / 4 * r * s - 9.0 / 8 * r * f2 * s);
  pb += (k1 - k2) * (3.0 / 8 * r2 * r * f + 3.0 / 8 * r * f2 * f - 3.0 / 8 * f2 * f * s - 3.0 / 8 * f * s2 * s -
                     1.0 / 4 * f2 * f - 3.0 / 4 * r2 * f - 3.0 / 4 * f * s2 + 1.0 / 4 * r * f - 1.0 / 4 * f * s +
                     9.0 / 8 * r * f * s2 - 9.0 / 8 * r2 * f * s + 3.0 / 2 * r * f * s);
  pb += 0.25 * (k1 + k2 - 8.0 * k3) * s2 * s + (k1 + k2 + 16.0 * k3) * (3.0 / 32 * s2 * s2 + 1.0 / 32 * s2);
  pb += 3.0 / 32 * (k1 + k2) * s2;  // the Gibbs-Duhem term missing from the print
  return pb;
}

// Pressure tensor of App. A at every cell, [6][N] in the order xx, yy, zz,
// xy, xz, yz, from the lattice gradients and Laplacians of rho, phi, psi.
// Mixing coefficients: k_rr = k_ff = (k1 + k2)/4, k_ss = (k1 + k2 + 4 k3)/4,
// k_rf = -k_fs = (k1 - k2)/4, k_rs = -(k1 + k2)/4.  Each cross pair (a, b)
// contributes d_a a d_b b + d_a b d_b a - (grad a . grad b) delta
// - a lap b delta - b lap a delta (the printed last pair reads psi (d_gg)
// for psi (d_gg phi), a typo).
void pressure_tensor(const Sim& s, std::vector<double>& P) {
  const long N = s.N;
  const double a2 = s.p.alpha * s.p.alpha;
  const double k1 = s.p.kappa1, k2 = s.p.kappa2, k3 = s.p.kappa3;
  // coefficient matrix over (rho, phi, psi)
  const double K[3][3] = {{(k1 + k2) / 4, (k1 - k2) / 4, -(k1 + k2) / 4},
                          {(k1 - k2) / 4, (k1 + k2) / 4, -(k1 - k2) / 4},
                          {-(k1 + k2) / 4, -(k1 - k2) / 4, (k1 + k2 + 4 * k3) / 4}};
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  P.assign(6 * N, 0.0);
  const std::vector<double>* fld[3] = {&s.rho, &s.phi, &s.psi};
#pragma omp parallel for
  for (long c = 0; c < N; ++c) {
    double g[3][3], L[3], v[3];
    for (int q = 0; q < 3; ++q) {
      grad(s, *fld[q], c, g[q]);
      L[q] = lap(s, *fld[q], c);
      v[q] = (*fld[q])[c];
    }
    double tr = bulk_pressure(s.p, v[0], v[1], v[2]);
    // isotropic part of the gradient terms: sum_ab K_ab (-(1/2) grad a . grad b - a lap b)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double gg = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
        tr += a2 * K[a][b] * (-0.5 * gg - v[a] * L[b]);
      }
    for (int q = 0; q < 6; ++q) {
      double t = ia[q] == ib[q] ? tr : 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) t += a2 * K[a][b] * g[a][ia[q]] * g[b][ib[q]];
      P[(long)q * N + c] = t;
    }
  }
}

// The free-energy force f_FE at every cell, [N][3], from the moment fields
// and the potentials of the step.
//  * potential form (the default): -rho grad mu~rho - phi grad mu_phi
//    - psi grad mu_psi' (eq. ForceFE with eq. GradPT; grad rho cs^2 cancels
//    rho grad cs^2 ln rho, so both ideal-gas parts are dropped).
//  * pressure-tensor form: grad(rho cs^2) - div p (App. A)
//    - psi grad(kappa_c (psi - I)), the first line of eq. ForceFE literally.
// The two agree in the continuum and differ at second order in the lattice
// spacing.
void fe_force(const Sim& s, std::vector<double>& F) {
  const long N = s.N;
  F.assign(3 * N, 0.0);
  if (s.p.force_form == 1) {
    std::vector<double> P, cpl(N);
    pressure_tensor(s, P);
    for (long c = 0; c < N; ++c) cpl[c] = s.p.kappa_c * (s.psi[c] - s.I[c]);
    std::vector<double> comp[6];
    for (int q = 0; q < 6; ++q) comp[q].assign(P.begin() + (long)q * N, P.begin() + (long)(q + 1) * N);
    // row a of the symmetric tensor: (xx, xy, xz), (xy, yy, yz), (xz, yz, zz)
    const int row[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma omp parallel for
    for (long c = 0; c < N; ++c) {
      double gr[3], gc[3], gp[3];
      grad(s, s.rho, c, gr);
      grad(s, cpl, c, gc);
      for (int a = 0; a < 3; ++a) {
        double div = 0.0;
        for (int b = 0; b < 3; ++b) {
          grad(s, comp[row[a][b]], c, gp);
          div += gp[b];
        }
        if (a < s.dim) F[3 * c + a] = CS2 * gr[a] - div - s.psi[c] * gc[a];
      }
    }
    return;
  }
#pragma omp parallel for
  for (long c = 0; c < N; ++c) {
    double gr[3], gp[3], gs[3];
    grad(s, s.mur, c, gr);
    grad(s, s.muphi, c, gp);
    grad(s, s.mupsi, c, gs);
    for (int k = 0; k < s.dim; ++k) F[3 * c + k] = -s.rho[c] * gr[k] - s.phi[c] * gp[k] - s.psi[c] * gs[k];
  }
}

std::vector<const double*> node_ptrs(const Sim& s) {
  std::vector<const double*> Xs;
  for (const Membrane& m : s.mem) Xs.push_back(m.X.data());
  return Xs;
}

void do_step(Sim& s) {
  const Lattice& L = s.L;
  const int Q = L.Q;
  const long N = s.N;
  // (1) moments at time t (eq. MomentsDFs)
  moments(s);
  // (2) membrane profile I from X(t) (eq. Iprofile)
  std::vector<const double*> Xs = node_ptrs(s);
  iprofile(s, Xs, s.I, s.dsel, s.band);
  // (3) chemical potentials (App. A) with mu_psi' (Sec. 3.1)
  potentials(s);
  // (4) membrane forces F_s + F_b + F_c at X(t) (eq. MembraneForces)
  std::vector<std::vector<double>> Fm(s.mem.size());
  for (size_t mi = 0; mi < s.mem.size(); ++mi) {
    Fm[mi].assign(3 * s.mem[mi].nn, 0.0);
    elastic_force(s.mem[mi], s.mem[mi].X.data(), Fm[mi].data());
  }
  coupling_force(s, Xs, s.band, s.psi, s.I, Fm);
  // (5) spreading to the lattice (eq. Spreading)
  spread(s, Xs, Fm, s.fib);
  // (6) total force: f_FE (potential form, or the pressure-tensor form when
  //     selected) plus f_IB
  s.F.assign(3 * N, 0.0);
  std::vector<double> ffe;
  fe_force(s, ffe);
#pragma omp parallel for
  for (long c = 0; c < N; ++c)
    for (int k = 0; k < s.dim; ++k) s.F[3 * c + k] = ffe[3 * c + k] + s.fib[3 * c + k];
  // (7) collision (eq. LBE): BGK + exact difference method for f (or Guo
  //     forcing when selected); BGK for g, h
  std::vector<double> fp(Q * N), gp(Q * N), hp(Q * N);
#pragma omp parallel for
  for (long c = 0; c < N; ++c) {
    double r = s.rho[c];
    double u[3], du[3], v[3], ud[3];
    for (int k = 0; k < 3; ++k) {
      u[k] = s.j[3 * c + k] / r;        // bare velocity, eq. MomentsDFs
      du[k] = s.F[3 * c + k] / r;       // eq. VelCorrection
      v[k] = u[k] + 0.5 * du[k];        // eq. ActualFluidVel
      ud[k] = u[k] + du[k];
    }
    double ge[19], he[19];
    oeq(L, s.phi[c], s.p.gamma_phi, s.muphi[c], v, ge);
    oeq(L, s.psi[c], s.p.gamma_psi, s.mupsi[c], v, he);
    const double* Fc = &s.F[3 * c];
    const double vF = v[0] * Fc[0] + v[1] * Fc[1] + v[2] * Fc[2];
    for (int i = 0; i < Q; ++i) {
      long k = (long)i * N + c;
      if (s.p.forcing == 1) {
        // Guo, Zheng and Shi (2002): BGK towards f^eq(rho, v), v = (j + F/2)/rho,
        // plus the source (1 - 1/(2 tau)) w_i [(c_i - v)/cs^2 + (c_i.v) c_i/cs^4] . F
        const double cv = cdot(L, i, v), cF = cdot(L, i, Fc);
        const double Si = (1.0 - 0.5 / s.p.tau) * L.w[i] * ((cF - vF) / CS2 + cv * cF / (CS2 * CS2));
        fp[k] = s.f[k] - (s.f[k] - feq(L, i, r, v)) / s.p.tau + Si;
      } else {
        double fe = feq(L, i, r, u);
        fp[k] = s.f[k] - (s.f[k] - fe) / s.p.tau + feq(L, i, r, ud) - fe;
      }
      gp[k] = s.g[k] - (s.g[k] - ge[i]) / s.p.tau_phi;
      hp[k] = s.h[k] - (s.h[k] - he[i]) / s.p.tau_psi;
    }
  }
  // (8) streaming f_i(x + c_i, t + 1) = f_i*(x): pull form, periodic, and
  //     halfway bounce-back at walls (zero normal velocity and flux, eq.
  //     NaturalBCs).  Reading: walls sit half a cell outside the first and
  //     last lattice planes.
#pragma omp parallel for
  for (long c = 0; c < N; ++c) {
    int x[3];
    ccoords(s, c, x);
    for (int i = 0; i < Q; ++i) {
      int q[3];
      bool bounce = false;
      for (int a = 0; a < 3; ++a) {
        int v = x[a] - L.c[i][a];
        if (is_wall_axis(s, a)) {
          if (v < 0 || v >= s.n[a]) bounce = true;
        } else {
          v = wrapi(v, s.n[a]);
        }
        q[a] = v;
      }
      long k = (long)i * N + c;
      if (bounce) {
        long kb = (long)L.opp[i] * N + c;
        s.f[k] = fp[kb];
        s.g[k] = gp[kb];
        s.h[k] = hp[kb];
      } else {
        long src = (long)i * N + cidx(s, q[0], q[1], q[2]);
        s.f[k] = fp[src];
        s.g[k] = gp[src];
        s.h[k] = hp[src];
      }
    }
  }
  // (9) interpolation and advection (eqs. Interpolation, UpdatedXl).
  //     Reading: v(t + dt) is taken from the streamed populations with the
  //     half-force correction of the force just applied, v' = (j' + F/2)/rho'.
  std::vector<double> vnew(3 * N, 0.0);
#pragma omp parallel for
  for (long c = 0; c < N; ++c) {
    double r = 0, jj[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      double fi = s.f[(long)i * N + c];
      r += fi;
      for (int k = 0; k < 3; ++k) jj[k] += L.c[i][k] * fi;
    }
    for (int k = 0; k < s.dim; ++k) vnew[3 * c + k] = (jj[k] + 0.5 * s.F[3 * c + k]) / r;
  }
  for (size_t mi = 0; mi < s.mem.size(); ++mi) {
    Membrane& m = s.mem[mi];
    std::vector<double> U(3 * m.nn);
    interp(s, m.X.data(), m.nn, vnew, U.data());
    for (int l = 0; l < m.nn; ++l)
      for (int k = 0; k < s.dim; ++k) m.X[3 * l + k] += U[3 * l + k];
  }
  emulate_storage(s);
  s.t += 1;
}

// Initial state.  The paper does not print one; reading: rho = 1 and u = u0,
// psi = I(X0), a flat C1/C2 interface s = (1 + tanh((z - z0)/(2 alpha)))/2
// along the last axis (eq. CmProfile) with C1 = (1 - psi) s, C2 = (1 - psi)(1 - s),
// and populations at equilibrium with the chemical potentials of these
// fields and no force.
void do_init(Sim& s, const double* C, const double* u) {
  const long N = s.N;
  std::vector<const double*> Xs = node_ptrs(s);
  iprofile(s, Xs, s.I, s.dsel, s.band);
  s.rho.assign(N, 1.0);
  s.phi.assign(N, 0.0);
  s.psi.assign(N, 0.0);
  s.j.assign(3 * N, 0.0);
  std::vector<double> uu(3 * N, 0.0);
  for (long c = 0; c < N; ++c) {
    if (C) {
      double c1 = C[c], c2 = C[N + c], c3 = C[2 * N + c];
      s.rho[c] = c1 + c2 + c3;
      s.phi[c] = c1 - c2;
      s.psi[c] = c3;
    } else {
      int x[3];
      ccoords(s, c, x);
      double z = x[s.dim - 1];
      double sv = 0.5 * (1.0 + std::tanh((z - s.p.interface_pos) / (2.0 * s.p.alpha)));
      if (s.p.interface_pos < 0) sv = 0.0;  // no interface: all C2 outside the capsules
      double ps = s.I[c];
      s.psi[c] = ps;
      s.phi[c] = (1.0 - ps) * (2.0 * sv - 1.0);
    }
    if (u) {
      for (int k = 0; k < 3; ++k) uu[3 * c + k] = (k < s.dim) ? u[k * N + c] : 0.0;
    } else {
      uu[3 * c] = s.p.u0x;
      uu[3 * c + 1] = s.p.u0y;
      uu[3 * c + 2] = (s.dim == 3) ? s.p.u0z : 0.0;
    }
  }
  potentials(s);
  const int Q = s.L.Q;
  s.f.assign(Q * N, 0.0);
  s.g.assign(Q * N, 0.0);
  s.h.assign(Q * N, 0.0);
  for (long c = 0; c < N; ++c) {
    double ge[19], he[19];
    oeq(s.L, s.phi[c], s.p.gamma_phi, s.muphi[c], &uu[3 * c], ge);
    oeq(s.L, s.psi[c], s.p.gamma_psi, s.mupsi[c], &uu[3 * c], he);
    for (int i = 0; i < Q; ++i) {
      s.f[(long)i * N + c] = feq(s.L, i, s.rho[c], &uu[3 * c]);
      s.g[(long)i * N + c] = ge[i];
      s.h[(long)i * N + c] = he[i];
    }
  }
  s.F.assign(3 * N, 0.0);
  emulate_storage(s);
  s.t = 0;
}

}  // namespace

// =================================================================== C API
extern "C" {

void* or_create(const or_params* p) {
  Sim* s = new Sim();
  s->p = *p;
  s->dim = p->dim;
  s->L = (p->dim == 2) ? make_d2q9() : make_d3q19();
  s->n[0] = p->nx;
  s->n[1] = p->ny;
  s->n[2] = (p->dim == 2) ? 1 : p->nz;
  s->N = (long)s->n[0] * s->n[1] * s->n[2];
  s->t = 0;
  return s;
}
void or_destroy(void* h) { delete (Sim*)h; }
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
int or_Q(void* h) { return ((Sim*)h)->L.Q; }
void or_lattice(void* h, int* c, double* w) {
  Sim* s = (Sim*)h;
  for (int i = 0; i < s->L.Q; ++i) {
    for (int k = 0; k < 3; ++k) c[3 * i + k] = s->L.c[i][k];
    w[i] = s->L.w[i];
  }
}

// kind 0: ring (X: n*3, consecutive markers joined); kind 1: triangles.
int or_add_membrane(void* h, int kind, int nn, const double* X, int ne, const int* E,
                    double ks, double kb, double G, double C) {
  Sim* s = (Sim*)h;
  Membrane m;
  m.kind = kind;
  m.nn = nn;
  m.ne = ne;
  m.X.assign(X, X + 3 * nn);
  if (kind == 1) m.E.assign(E, E + 3 * ne);
  m.ks = ks;
  m.kb = kb;
  m.G = G;
  m.C = C;
  membrane_setup(m);
  s->mem.push_back(m);
  return (int)s->mem.size() - 1;
}

void or_init(void* h, const double* C, const double* u) { do_init(*(Sim*)h, C, u); }
void or_step(void* h, int n) {
  for (int k = 0; k < n; ++k) do_step(*(Sim*)h);
}
long or_time(void* h) { return ((Sim*)h)->t; }

// populations as [set][i][cell] (set 0 f, 1 g, 2 h)
void or_get_pops(void* h, double* out) {
  Sim* s = (Sim*)h;
  long QN = (long)s->L.Q * s->N;
  std::memcpy(out, s->f.data(), QN * sizeof(double));
  std::memcpy(out + QN, s->g.data(), QN * sizeof(double));
  std::memcpy(out + 2 * QN, s->h.data(), QN * sizeof(double));
}
void or_set_pops(void* h, const double* in) {
  Sim* s = (Sim*)h;
  long QN = (long)s->L.Q * s->N;
  s->f.assign(in, in + QN);
  s->g.assign(in + QN, in + 2 * QN);
  s->h.assign(in + 2 * QN, in + 3 * QN);
}
void or_get_nodes(void* h, int m, double* X) {
  Sim* s = (Sim*)h;
  std::memcpy(X, s->mem[m].X.data(), s->mem[m].X.size() * sizeof(double));
}
void or_set_nodes(void* h, int m, const double* X) {
  Sim* s = (Sim*)h;
  std::memcpy(s->mem[m].X.data(), X, s->mem[m].X.size() * sizeof(double));
}

// Fields of the current populations: 0 rho, 1 phi, 2 psi, 3-5 bare u,
// 6 C1, 7 C2, 8 C3; of the last step: 9 I, 10-12 total force, 13-15 f_IB,
// 16 mu~rho, 17 mu_phi, 18 mu_psi'.
void or_get_field(void* h, int which, double* out) {
  Sim* s = (Sim*)h;
  const long N = s->N;
  if (which <= 8) {
    std::vector<double> keep_rho = s->rho, keep_phi = s->phi, keep_psi = s->psi, keep_j = s->j;
    moments(*s);
    for (long c = 0; c < N; ++c) {
      double r = s->rho[c], ph = s->phi[c], ps = s->psi[c];
      double v = 0;
      switch (which) {
        case 0: v = r; break;
        case 1: v = ph; break;
        case 2: v = ps; break;
        case 3: case 4: case 5: v = s->j[3 * c + which - 3] / r; break;
        case 6: v = 0.5 * (r + ph - ps); break;
        case 7: v = 0.5 * (r - ph - ps); break;
        case 8: v = ps; break;
      }
      out[c] = v;
    }
    s->rho = keep_rho; s->phi = keep_phi; s->psi = keep_psi; s->j = keep_j;
    return;
  }
  for (long c = 0; c < N; ++c) {
    double v = 0;
    if (which == 9) v = s->I.empty() ? 0 : s->I[c];
    else if (which >= 10 && which <= 12) v = s->F.empty() ? 0 : s->F[3 * c + which - 10];
    else if (which >= 13 && which <= 15) v = s->fib.empty() ? 0 : s->fib[3 * c + which - 13];
    else if (which == 16) v = s->mur.empty() ? 0 : s->mur[c];
    else if (which == 17) v = s->muphi.empty() ? 0 : s->muphi[c];
    else if (which == 18) v = s->mupsi.empty() ? 0 : s->mupsi[c];
    out[c] = v;
  }
}

// ------------------------------------------------ pieces exposed for pins
double or_peskin(double r) { return peskin(r); }
double or_round(double x, int p, int emin, double maxv) { return round_to_format(x, p, emin, maxv); }

// which: 0 stretching (2D) / Skalak (3D); 1 bending (2D) / Helfrich (3D)
double or_mem_energy(void* h, int m, int which, const double* X) {
  const Membrane& mm = ((Sim*)h)->mem[m];
  if (mm.kind == 0) return which == 0 ? ring_stretch_energy(mm, X) : ring_bend_energy(mm, X);
  if (which == 0) return skalak_energy(mm, X);
  double E;
  helfrich_eval(mm, X, &E, nullptr);
  return E;
}
void or_mem_force(void* h, int m, int which, const double* X, double* F) {
  const Membrane& mm = ((Sim*)h)->mem[m];
  std::memset(F, 0, 3 * mm.nn * sizeof(double));
  if (mm.kind == 0) {
    if (which == 0) ring_stretch_force(mm, X, F); else ring_bend_force(mm, X, F);
  } else {
    if (which == 0) skalak_force(mm, X, F); else helfrich_eval(mm, X, nullptr, F);
  }
}

// Membrane profile for given marker positions (concatenated over membranes).
// Returns the number of band cells.
long or_iprofile(void* h, const double* Xall, double* I, double* d) {
  Sim* s = (Sim*)h;
  std::vector<const double*> Xs;
  long off = 0;
  for (const Membrane& m : s->mem) { Xs.push_back(Xall + off); off += 3 * m.nn; }
  std::vector<double> Iv, dv;
  std::vector<BandCell> band;
  iprofile(*s, Xs, Iv, dv, band);
  if (I) std::memcpy(I, Iv.data(), s->N * sizeof(double));
  if (d) std::memcpy(d, dv.data(), s->N * sizeof(double));
  return (long)band.size();
}

// Coupling energy (eq. DiscreteCE) for a given psi field and marker positions;
// writes the coupling force on every marker (concatenated) when F != NULL.
double or_coupling(void* h, const double* psi, const double* Xall, double* F) {
  Sim* s = (Sim*)h;
  std::vector<const double*> Xs;
  long off = 0;
  for (const Membrane& m : s->mem) { Xs.push_back(Xall + off); off += 3 * m.nn; }
  std::vector<double> Iv, dv;
  std::vector<BandCell> band;
  iprofile(*s, Xs, Iv, dv, band);
  std::vector<double> ps(psi, psi + s->N);
  double E = 0.0;
  for (long c = 0; c < s->N; ++c) E += 0.5 * s->p.kappa_c * (ps[c] - Iv[c]) * (ps[c] - Iv[c]);
  if (F) {
    std::vector<std::vector<double>> Fm(s->mem.size());
    for (size_t mi = 0; mi < s->mem.size(); ++mi) Fm[mi].assign(3 * s->mem[mi].nn, 0.0);
    coupling_force(*s, Xs, band, ps, Iv, Fm);
    long o = 0;
    for (size_t mi = 0; mi < s->mem.size(); ++mi) {
      std::memcpy(F + o, Fm[mi].data(), Fm[mi].size() * sizeof(double));
      o += Fm[mi].size();
    }
  }
  return E;
}

// Chemical potentials (mu~rho, mu_phi, mu_psi') of given fields.
void or_potentials(void* h, const double* rho, const double* phi, const double* psi,
                   const double* I, double* mur, double* mup, double* mus) {
  Sim* s = (Sim*)h;
  s->rho.assign(rho, rho + s->N);
  s->phi.assign(phi, phi + s->N);
  s->psi.assign(psi, psi + s->N);
  s->I.assign(I, I + s->N);
  potentials(*s);
  std::memcpy(mur, s->mur.data(), s->N * sizeof(double));
  std::memcpy(mup, s->muphi.data(), s->N * sizeof(double));
  std::memcpy(mus, s->mupsi.data(), s->N * sizeof(double));
}

// Spreading of given nodal forces (concatenated) at given positions.
void or_spread(void* h, const double* Xall, const double* Fall, double* fib) {
  Sim* s = (Sim*)h;
  std::vector<const double*> Xs;
  std::vector<std::vector<double>> F;
  long off = 0;
  for (const Membrane& m : s->mem) {
    Xs.push_back(Xall + off);
    F.emplace_back(Fall + off, Fall + off + 3 * m.nn);
    off += 3 * m.nn;
  }
  std::vector<double> out;
  spread(*s, Xs, F, out);
  for (long c = 0; c < s->N; ++c)
    for (int k = 0; k < 3; ++k) fib[k * s->N + c] = out[3 * c + k];
}
// Interpolation of a given vector field [3][N] at given positions (one membrane).
void or_interp(void* h, int nn, const double* X, const double* field, double* U) {
  Sim* s = (Sim*)h;
  std::vector<double> v(3 * s->N);
  for (long c = 0; c < s->N; ++c)
    for (int k = 0; k < 3; ++k) v[3 * c + k] = field[k * s->N + c];
  interp(*s, X, nn, v, U);
}

// Lattice gradient ([3][N]) and Laplacian of a given scalar field, the
// isotropic stencils of the step (periodic, mirror ghost at walls).
void or_grad_field(void* h, const double* a, double* g) {
  Sim* s = (Sim*)h;
  std::vector<double> av(a, a + s->N);
  for (long c = 0; c < s->N; ++c) {
    double gg[3];
    grad(*s, av, c, gg);
    for (int k = 0; k < 3; ++k) g[k * s->N + c] = gg[k];
  }
}
void or_lap_field(void* h, const double* a, double* out) {
  Sim* s = (Sim*)h;
  std::vector<double> av(a, a + s->N);
  for (long c = 0; c < s->N; ++c) out[c] = lap(*s, av, c);
}

// Free-energy force f_FE ([3][N]) of given fields, exactly as the step forms
// it (potential form or pressure-tensor form per the parameters, with
// mu_psi' from I), without the immersed-boundary part.
void or_force_fe(void* h, const double* rho, const double* phi, const double* psi, const double* I,
                 double* F) {
  Sim* s = (Sim*)h;
  s->rho.assign(rho, rho + s->N);
  s->phi.assign(phi, phi + s->N);
  s->psi.assign(psi, psi + s->N);
  s->I.assign(I, I + s->N);
  potentials(*s);
  std::vector<double> f;
  fe_force(*s, f);
  for (long c = 0; c < s->N; ++c)
    for (int k = 0; k < 3; ++k) F[k * s->N + c] = f[3 * c + k];
}
double or_bulk_pressure(void* h, double rho, double phi, double psi) {
  return bulk_pressure(((Sim*)h)->p, rho, phi, psi);
}

// Shape measures of membrane m at positions X (unwrapped markers):
// out[0] = area, out[1] = volume.  2D ring: the enclosed area by the
// shoelace formula (volume 0).  3D: the sum of the triangle areas, and the
// enclosed volume by the divergence theorem, sum over triangles of
// a . (b x c) / 6 (positive for triangles counter-clockwise seen from
// outside).
void or_capsule_measures(void* h, int m, const double* X, double* out) {
  const Membrane& mm = ((Sim*)h)->mem[m];
  double A = 0.0, V = 0.0;
  if (mm.kind == 0) {
    for (int l = 0; l < mm.nn; ++l) {
      const double* p = &X[3 * l];
      const double* q = &X[3 * ((l + 1) % mm.nn)];
      A += 0.5 * (p[0] * q[1] - q[0] * p[1]);
    }
  } else {
    for (int t = 0; t < mm.ne; ++t) {
      const double* a = &X[3 * mm.E[3 * t]];
      const double* b = &X[3 * mm.E[3 * t + 1]];
      const double* c = &X[3 * mm.E[3 * t + 2]];
      double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      A += 0.5 * n3(cr);
      double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
      V += (a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]) / 6.0;
    }
  }
  out[0] = A;
  out[1] = V;
}

// Interpolation of a scalar lattice field at one point with the kernel of
// eq. DiscreteDirac (as eq. Interpolation does for the velocity).
static double interp_scalar(const Sim& s, const double* P, const std::vector<double>& a) {
  int base[3] = {0, 0, 0}, span[3] = {1, 1, 1};
  for (int k = 0; k < s.dim; ++k) { base[k] = (int)std::floor(P[k]) - 1; span[k] = 4; }
  double acc = 0.0;
  for (int i0 = 0; i0 < span[0]; ++i0)
    for (int i1 = 0; i1 < span[1]; ++i1)
      for (int i2 = 0; i2 < span[2]; ++i2) {
        int q[3] = {base[0] + i0, base[1] + i1, base[2] + i2};
        double wgt = 1.0;
        for (int k = 0; k < s.dim; ++k) wgt *= peskin(q[k] - P[k]);
        if (wgt == 0.0) continue;
        bool out = false;
        for (int k = 0; k < 3; ++k) {
          if (is_wall_axis(s, k)) { if (q[k] < 0 || q[k] >= s.n[k]) out = true; }
          else q[k] = wrapi(q[k], s.n[k]);
        }
        if (out) continue;
        acc += wgt * a[cidx(s, q[0], q[1], q[2])];
      }
  return acc;
}

// Contact angle of membrane m (positions X) with the C1/C2 interface
// phi = C1 - C2 = 0, the equilibrium measure of the capsule at a
// fluid-fluid interface (Sec. 4.1).  The paper prints no discrete recipe;
// reading: phi is interpolated to the markers with the kernel of eq.
// DiscreteDirac; every membrane edge whose end values change sign holds a
// contact point at the linear zero crossing; there the interface normal is
// the interpolated lattice gradient of phi (pointing into C1) and the
// membrane normal is the linear interpolation along the edge of its two
// end markers' outward normals (a marker's normal: the normalised sum of
// the area vectors of its triangles in 3D, of the outward normals of its
// two segments in 2D).  The angle at a contact point is the angle between
// the two unit normals; the result is their mean in degrees.  out[0] =
// mean, out[1] = smallest, out[2] = largest angle.  Returns the number of
// contact points (0: the membrane does not cross the interface; out is
// then left unchanged).
int or_contact_angle(void* h, int m, const double* X, const double* phi, double* out) {
  Sim* s = (Sim*)h;
  const Membrane& mm = s->mem[m];
  const long N = s->N;
  std::vector<double> ph(phi, phi + N), g[3];
  for (int k = 0; k < 3; ++k) g[k].assign(N, 0.0);
  for (long c = 0; c < N; ++c) {
    double gg[3];
    grad(*s, ph, c, gg);
    for (int k = 0; k < 3; ++k) g[k][c] = gg[k];
  }
  std::vector<double> pn(mm.nn);
  for (int l = 0; l < mm.nn; ++l) pn[l] = interp_scalar(*s, &X[3 * l], ph);
  // marker normals and the edges
  std::vector<double> vn(3 * mm.nn, 0.0);
  std::vector<int> ea, eb;
  if (mm.kind == 0) {
    for (int l = 0; l < mm.nn; ++l) {
      int l1 = (l + 1) % mm.nn;
      double tx = X[3 * l1] - X[3 * l], ty = X[3 * l1 + 1] - X[3 * l + 1];
      double lt = std::sqrt(tx * tx + ty * ty);
      for (int q : {l, l1}) {
        vn[3 * q] += ty / lt;
        vn[3 * q + 1] += -tx / lt;
      }
      ea.push_back(l);
      eb.push_back(l1);
    }
  } else {
    std::vector<std::pair<int, int>> edges;
    for (int t = 0; t < mm.ne; ++t) {
      const int* v = &mm.E[3 * t];
      const double* a = &X[3 * v[0]];
      const double* b = &X[3 * v[1]];
      const double* c = &X[3 * v[2]];
      double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      for (int q = 0; q < 3; ++q) {
        for (int k = 0; k < 3; ++k) vn[3 * v[q] + k] += cr[k];
        edges.push_back({std::min(v[q], v[(q + 1) % 3]), std::max(v[q], v[(q + 1) % 3])});
      }
    }
    std::sort(edges.begin(), edges.end());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    for (auto& e : edges) {
      ea.push_back(e.first);
      eb.push_back(e.second);
    }
  }
  for (int l = 0; l < mm.nn; ++l) {
    double len = n3(&vn[3 * l]);
    for (int k = 0; k < 3; ++k) vn[3 * l + k] /= len;
  }
  int cnt = 0;
  double sum = 0.0, lo = 1e300, hi = -1e300;
  for (size_t e = 0; e < ea.size(); ++e) {
    const double fa = pn[ea[e]], fb = pn[eb[e]];
    if (!(fa * fb < 0.0)) continue;
    const double t = fa / (fa - fb);
    double P[3], nm[3], gp[3];
    for (int k = 0; k < 3; ++k) {
      P[k] = X[3 * ea[e] + k] + t * (X[3 * eb[e] + k] - X[3 * ea[e] + k]);
      nm[k] = (1.0 - t) * vn[3 * ea[e] + k] + t * vn[3 * eb[e] + k];
    }
    for (int k = 0; k < 3; ++k) gp[k] = interp_scalar(*s, P, g[k]);
    const double lg = n3(gp), lm = n3(nm);
    if (!(lg > 0.0) || !(lm > 0.0)) continue;
    double cs = (gp[0] * nm[0] + gp[1] * nm[1] + gp[2] * nm[2]) / (lg * lm);
    cs = std::min(1.0, std::max(-1.0, cs));
    const double ang = std::acos(cs) * 180.0 / M_PI;
    sum += ang;
    lo = std::min(lo, ang);
    hi = std::max(hi, ang);
    ++cnt;
  }
  if (cnt > 0) {
    out[0] = sum / cnt;
    out[1] = lo;
    out[2] = hi;
  }
  return cnt;
}

// FP64 totals of the current populations: sum rho, sum phi, sum psi.  Cell
// sums are accumulated with Neumaier's compensated summation so that the
// totals resolve changes far below the rounding of a plain running sum.
void or_masses(void* h, double* out) {
  Sim* s = (Sim*)h;
  const int Q = s->L.Q;
  for (int set = 0; set < 3; ++set) {
    const std::vector<double>& P = set == 0 ? s->f : (set == 1 ? s->g : s->h);
    double sum = 0.0, comp = 0.0;
    for (long k = 0; k < s->N; ++k) {
      double cell = 0.0;
      for (int i = 0; i < Q; ++i) cell += P[(long)i * s->N + k];
      double t = sum + cell;
      if (std::fabs(sum) >= std::fabs(cell)) comp += (sum - t) + cell;
      else comp += (cell - t) + sum;
      sum = t;
    }
    out[set] = sum + comp;
  }
}

}  // extern "C"
