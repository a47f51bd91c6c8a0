// Equilibrium-quality read-out: the contact angle of every capsule with the
// C1/C2 interface phi = 0, in FP64 (Sec. 4.1 compares equilibrium shapes of
// a capsule at a fluid-fluid interface; the paper prints no discrete
// recipe for the angle).  Recipe of this library:
//  * phi (FP64 sums of the streamed populations) is interpolated to every
//    marker with the kernel of eq. DiscreteDirac;
//  * every membrane edge whose end values change sign holds a contact point
//    at the linear zero crossing;
//  * there, the interface normal is the delta_h-interpolated lattice
//    gradient of phi (the isotropic stencil, mirror ghost at walls) and the
//    membrane normal is the linear interpolation along the edge of the end
//    markers' outward normals (sum of the incident triangles' area vectors
//    in 3D; of the two segments' unit normals in 2D), normalised;
//  * the angle between the two unit normals, in degrees; per capsule the
//    mean over its contact points (summed in edge order), the smallest and
//    the largest.
// Diagnostic only: launched by tlb_contact_angle, never inside a step.
#pragma once
#include "tlb_common.cuh"
#include "tlb_ibm.cuh"

struct AngleArgs {
  Geo G;
  int dim, nn, NV;
  const double* X;      // [nn][3] unwrapped markers
  const double* phi;    // [N] FP64 phi
  const int* E;         // elements
  const int* inc_off;   // incidence CSR
  const int* inc;
  const int* rnext;     // 2D ring successor
  const int* rprev;
  const int* edges;     // 3D: [nedge][4] va, vb, face, face
  const int* ncap;      // capsule of each marker
  int nedge;            // edges: 3D nedge, 2D nn (segment l -> rnext[l])
  double* mk;           // [nn][4] phi and unit normal of each marker
  double* ang;          // [nedge] angle of the edge's contact point, or NaN
  int* ecapo;           // [nedge] capsule of the edge
};

__device__ __forceinline__ int wrap_or_clamp(int v, int n, bool wall) {
  if (wall) return v < 0 ? -1 : (v >= n ? -1 : v);
  v %= n;
  return v < 0 ? v + n : v;
}

// delta_h-weighted sum over the 4^d support cells of point P of a per-cell
// value fn(cell index); cells beyond a wall are skipped.
template <class Fn>
__device__ double support_sum(const Geo& G, int dim, const double* P, Fn fn) {
  int base[3], span[3] = {4, dim == 3 ? 4 : 1, 4};
  for (int d = 0; d < 3; ++d) base[d] = (int)floor(P[d]) - 1;
  if (dim == 2) base[1] = 0;
  double acc = 0.0;
  for (int oz = 0; oz < span[2]; ++oz)
    for (int oy = 0; oy < span[1]; ++oy)
      for (int ox = 0; ox < span[0]; ++ox) {
        const int q[3] = {base[0] + ox, base[1] + oy, base[2] + oz};
        double w = peskin<double>(q[0] - P[0]) * peskin<double>(q[2] - P[2]);
        if (dim == 3) w *= peskin<double>(q[1] - P[1]);
        if (w == 0.0) continue;
        const int x = wrap_or_clamp(q[0], G.nx, false);
        const int y = dim == 3 ? wrap_or_clamp(q[1], G.ny, false) : 0;
        const int z = wrap_or_clamp(q[2], G.nz, G.wall);
        if (z < 0) continue;
        acc += w * fn(((long long)z * G.ny + y) * G.nx + x, x, y, z);
      }
  return acc;
}

// Lattice gradient component d of phi at cell (x, y, z): (1/cs^2) sum_i
// w_i c_i phi(x + c_i), periodic, mirror ghost phi(-1) = phi(0) at walls.
template <class L>
__device__ double phi_grad(const Geo& G, const double* phi, int x, int y, int z, int d) {
  double g = 0.0;
#pragma unroll
  for (int i = 1; i < L::Q; ++i) {
    const int cd = d == 0 ? L::cx(i) : (d == 1 ? L::cy(i) : L::cz(i));
    if (cd == 0) continue;
    const int sx = wrapc(x + L::cx(i), G.nx), sy = wrapc(y + L::cy(i), G.ny);
    int sz = z + L::cz(i);
    sz = G.wall ? min(max(sz, 0), G.nz - 1) : wrapc(sz, G.nz);
    g += L::w(i) * cd * phi[((long long)sz * G.ny + sy) * G.nx + sx];
  }
  return 3.0 * g;
}

// phi and the outward unit normal at every marker.
static __global__ void k_marker_phi(AngleArgs a) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= a.nn) return;
  const double* P = a.X + 3 * l;
  const double f = support_sum(a.G, a.dim, P, [&](long long c, int, int, int) { return a.phi[c]; });
  double n[3] = {0, 0, 0};
  if (a.dim == 2) {
    // internal (x, z) is the paper's (x, y): outward normal (t_z, -t_x)
    const int nb[2] = {a.rprev[l], a.rnext[l]};
    for (int s = 0; s < 2; ++s) {
      const double* p = a.X + 3 * (s == 0 ? nb[0] : l);
      const double* q = a.X + 3 * (s == 0 ? l : nb[1]);
      const double tx = q[0] - p[0], tz = q[2] - p[2], lt = sqrt(tx * tx + tz * tz);
      n[0] += tz / lt;
      n[2] += -tx / lt;
    }
  } else {
    for (int k = a.inc_off[l]; k < a.inc_off[l + 1]; ++k) {
      const int* v = a.E + 3 * a.inc[k];
      const double* p0 = a.X + 3 * v[0];
      const double* p1 = a.X + 3 * v[1];
      const double* p2 = a.X + 3 * v[2];
      const double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
      const double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
      n[0] += e1[1] * e2[2] - e1[2] * e2[1];
      n[1] += e1[2] * e2[0] - e1[0] * e2[2];
      n[2] += e1[0] * e2[1] - e1[1] * e2[0];
    }
  }
  const double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  a.mk[4 * l] = f;
  for (int k = 0; k < 3; ++k) a.mk[4 * l + 1 + k] = n[k] / ln;
}

// The contact point of every edge that crosses phi = 0 and its angle.
template <class L>
__global__ void k_contact_edges(AngleArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.nedge) return;
  const int va = a.dim == 2 ? e : a.edges[4 * e];
  const int vb = a.dim == 2 ? a.rnext[e] : a.edges[4 * e + 1];
  a.ecapo[e] = a.ncap[va];
  double ang = nan("");
  const double fa = a.mk[4 * va], fb = a.mk[4 * vb];
  if (fa * fb < 0.0) {
    const double t = fa / (fa - fb);
    double P[3], nm[3], g[3];
    for (int k = 0; k < 3; ++k) {
      P[k] = a.X[3 * va + k] + t * (a.X[3 * vb + k] - a.X[3 * va + k]);
      nm[k] = (1.0 - t) * a.mk[4 * va + 1 + k] + t * a.mk[4 * vb + 1 + k];
    }
    for (int d = 0; d < 3; ++d)
      g[d] = (a.dim == 2 && d == 1)
                 ? 0.0
                 : support_sum(a.G, a.dim, P,
                               [&](long long, int x, int y, int z) { return phi_grad<L>(a.G, a.phi, x, y, z, d); });
    const double lg = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const double lm = sqrt(nm[0] * nm[0] + nm[1] * nm[1] + nm[2] * nm[2]);
    if (lg > 0.0 && lm > 0.0) {
      const double cs = fmin(1.0, fmax(-1.0, (g[0] * nm[0] + g[1] * nm[1] + g[2] * nm[2]) / (lg * lm)));
      ang = acos(cs) * (180.0 / 3.14159265358979323846);
    }
  }
  a.ang[e] = ang;
}

// Per capsule (one block each): sum, count, min and max of the edge angles.
// Each thread folds a fixed stride of edges, then a fixed tree: the result
// does not depend on scheduling.  out[cap] = {mean, min, max, count}.
static __global__ void k_contact_reduce(const double* ang, const int* ecapo, int nedge, double* out) {
  __shared__ double ssum[256], smin[256], smax[256], scnt[256];
  const int cap = blockIdx.x;
  double s = 0.0, lo = 1e300, hi = -1e300, n = 0.0;
  for (int e = threadIdx.x; e < nedge; e += blockDim.x) {
    const double v = ang[e];
    if (ecapo[e] != cap || !(v == v)) continue;
    s += v;
    lo = fmin(lo, v);
    hi = fmax(hi, v);
    n += 1.0;
  }
  ssum[threadIdx.x] = s;
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  scnt[threadIdx.x] = n;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      ssum[threadIdx.x] += ssum[threadIdx.x + k];
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + k]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + k]);
      scnt[threadIdx.x] += scnt[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double c = scnt[0];
    out[4 * cap] = c > 0 ? ssum[0] / c : nan("");
    out[4 * cap + 1] = c > 0 ? smin[0] : nan("");
    out[4 * cap + 2] = c > 0 ? smax[0] : nan("");
    out[4 * cap + 3] = c;
  }
}
