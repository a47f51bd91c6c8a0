// Immersed-boundary kernels: membrane profile I (eq. Iprofile), coupling
// force (eqs. DiscreteCE, DiscreteCF), elastic forces (2D: eqs. DiscreteSE,
// DiscreteBE; 3D: Skalak shear and Helfrich bending), spreading (eq.
// Spreading with eq. DiscreteDirac), interpolation and advection (eqs.
// Interpolation, UpdatedXl).
#pragma once
#include <type_traits>

#include "tlb_common.cuh"

constexpr unsigned long long KEY_NONE = ~0ull;
constexpr int BRICK = 4;  // spreading bins are 4x4x4 cells (4x1x4 in 2D)

template <class Real>
struct IBArgs {
  Geo G;
  int dim, NV;  // dim 2: segments (NV = 2); dim 3: triangles (NV = 3)
  int nn, ne;
  double* X;             // [nn][3] unwrapped positions
  int* xo;               // [nn][3] floor(X) (kept by the box and advection kernels)
  Real* xr;              // [nn][3] X - xo
  const int* E;          // [ne][NV]
  const int* ecap;       // element -> capsule
  const int* ncap;       // node -> capsule
  const double* ks;      // per capsule
  const double* kb;
  const double* sG;
  const double* sC;
  const double* ds0;     // 2D: rest length of segment e
  const int* rprev;      // 2D: previous node on the ring
  const int* rnext;      // 2D: next node on the ring
  const double* A0;      // 3D: reference area per triangle
  const double* G0i;     // 3D: inverse reference metric per triangle (3)
  const Real* skc;       // 3D: per triangle G0i[0], 2 G0i[1], G0i[2], det G0i, A0 (working precision)
  const Real* capr;      // per capsule ks, kb, G, C (working precision), [4][ncaps]
  int ncaps;
  const int* inc_off;    // node -> incident elements (CSR, ascending)
  const int* inc;
  const int* adj;        // 3D: triangle across edge q (q: vertex q -> q+1)
  const int* ring_off;   // node -> distinct 1-ring neighbours (CSR, in the order
  const int* ring;       // of the incident elements and their vertices)
  int nedge;             // 3D: unique edges
  const int* edges;      // 3D: [nedge][4] vertex a, vertex b, face left, face right
  // per-step work
  Real* en;              // [ne][3] unit outward normal
  Real* vn;              // [nn][3] angle-weighted vertex pseudo-normal
  Real* erel;            // [ne][NV][3] vertices relative to the element's origin
  int* eorg;             // [ne][3] element origin: floor of its first vertex
  Real* ecst;            // [ne][16] edge vectors ab, ac, bc, Gram entries d00 d01 d11 and
                         // the reciprocals of d00, d11, |bc|^2 and the Gram determinant
  unsigned long long* ncpl;  // [nn][3] coupling force per marker, fixed point (CPL_SCALE)
  Real* F;               // [nn][3] node force
  int* box;              // [6] marker box accumulator: floor(min X), -ceil(max X)
  const int* boxc;       // [6] the step's marker box (snapshot of the accumulator)
  unsigned long long* key;
  int* own;
  Real* I;
  Real* dsel;
  const Real* psi;       // psi(t) (moment field)
  const Real* M;         // moment storage: the stored moments the interpolation
                         // rebuilds the streamed populations from (NULL: the
                         // population buffers are read)
  Real* fib;             // [3][P]
  const Real* ftot;      // [3][P]
  int* bcnt;             // bricks: count, previous count, cursor, offset
  int* bprev;
  int* bcur;
  int* boff;
  int* blist;
  int* bact;             // active bricks (compacted list)
  unsigned char* bflag;  // per brick: markers spread into it this step
  int* ctr;              // [0] active bricks, [1] list slots claimed
  int nbx, nby, nbz, nbricks;
  Real alpha, dc, kc;
  Real Iin, Iout;        // I beyond dc inside / outside: (1 +- tanh(dc/(2 alpha)))/2
  unsigned* status;
};

// ------------------------------------------------------------ small vectors
template <class T> struct V3 { T x, y, z; };
template <class T> TLB_HD V3<T> mk(T a, T b, T c) { return {a, b, c}; }
template <class T> TLB_HD V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> TLB_HD V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> TLB_HD V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> TLB_HD T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> TLB_HD V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Correctly rounded reciprocal (the value of 1 / x, without the division).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// Marker coordinates in the working precision.  FP32 builds them from the
// split X = xo + xr (integer cell, fraction) so that the per-step kernels
// issue no FP64 instructions (a slow pipe on this GPU); FP64 subtracts the
// positions directly.
// X_j - X_k along axis d:
template <class Real>
__device__ __forceinline__ Real node_dx(const IBArgs<Real>& a, int j, int k, int d) {
  if constexpr (std::is_same<Real, float>::value)
    return (float)(a.xo[3 * j + d] - a.xo[3 * k + d]) + (a.xr[3 * j + d] - a.xr[3 * k + d]);
  else
    return a.X[3 * j + d] - a.X[3 * k + d];
}
template <class Real>
__device__ __forceinline__ V3<Real> node_dv(const IBArgs<Real>& a, int j, int k) {
  return mk<Real>(node_dx(a, j, k, 0), node_dx(a, j, k, 1), node_dx(a, j, k, 2));
}
// X_l - o along axis d for an integer o:
template <class Real>
__device__ __forceinline__ Real node_off(const IBArgs<Real>& a, int l, int d, int o) {
  if constexpr (std::is_same<Real, float>::value)
    return (float)(a.xo[3 * l + d] - o) + a.xr[3 * l + d];
  else
    return a.X[3 * l + d] - (double)o;
}
// the split of one coordinate (clamped like the marker box)
template <class Real>
__device__ __forceinline__ void split_coord(double x, int* xo, Real* xr) {
  const double v = fmax(-1e8, fmin(1e8, x));
  const double f = floor(v);
  *xo = (int)f;
  *xr = (Real)(v - f);
}

// Closest point of cell p (unwrapped) on element e, relative to the cell,
// its barycentric weights and feature (0 interior, 1..3 edge starting at
// vertex feat-1, 4..6 vertex feat-4), without branches: the plane projection when it falls inside the face, else the
// nearest of the three clamped edge projections (ties to the first edge).
// The vertices come from the step's element-relative copy (erel, eorg) and
// the edge constants from ecst, so a cell needs no division and no
// double-precision arithmetic.
template <class Real>
__device__ __forceinline__ V3<Real> elem_closest(const IBArgs<Real>& a, int e, const int* p, Real* beta, int* feat) {
  const Real* r = a.erel + 3 * a.NV * e;
  const int* o = a.eorg + 3 * e;
  const Real* k = a.ecst + 16 * e;
  const V3<Real> A = mk<Real>(r[0] + (Real)(o[0] - p[0]), r[1] + (Real)(o[1] - p[1]), r[2] + (Real)(o[2] - p[2]));
  const V3<Real> ab = mk<Real>(k[0], k[1], k[2]);
  const V3<Real> ap = mk<Real>(-A.x, -A.y, -A.z);
  const Real d20 = dot(ap, ab);
  const Real t0 = fmin(Real(1), fmax(Real(0), d20 * k[12]));
  const V3<Real> P0 = A + t0 * ab;
  const int f0 = t0 <= Real(0) ? 4 : (t0 >= Real(1) ? 5 : 1);
  if (a.NV == 2) {
    beta[0] = Real(1) - t0;
    beta[1] = t0;
    beta[2] = 0;
    *feat = f0 == 1 ? 0 : f0;  // a segment's interior is its face
    return P0;
  }
  const V3<Real> ac = mk<Real>(k[3], k[4], k[5]), bc = mk<Real>(k[6], k[7], k[8]);
  const Real d00 = k[9], d01 = k[10], d11 = k[11];
  const Real d21 = dot(ap, ac);
  const Real t1 = fmin(Real(1), fmax(Real(0), d21 * k[13]));
  const V3<Real> P1 = A + t1 * ac;
  const V3<Real> Bv = A + ab;
  const Real t2 = fmin(Real(1), fmax(Real(0), -dot(Bv, bc) * k[14]));
  const V3<Real> P2 = Bv + t2 * bc;
  const Real D0 = dot(P0, P0), D1 = dot(P1, P1), D2 = dot(P2, P2);
  const Real v = (d11 * d20 - d01 * d21) * k[15], w = (d00 * d21 - d01 * d20) * k[15];
  const bool inside = k[15] > Real(0) && v >= Real(0) && w >= Real(0) && v + w <= Real(1);
  if (inside) {
    beta[0] = Real(1) - v - w;
    beta[1] = v;
    beta[2] = w;
    *feat = 0;
    return A + v * ab + w * ac;
  }
  const bool e1 = D1 < D0 && D1 <= D2, e2 = !e1 && D2 < D0;
  if (e2) {
    beta[0] = 0;
    beta[1] = Real(1) - t2;
    beta[2] = t2;
    *feat = t2 <= Real(0) ? 5 : (t2 >= Real(1) ? 6 : 2);
    return P2;
  }
  if (e1) {
    beta[0] = Real(1) - t1;
    beta[1] = 0;
    beta[2] = t1;
    *feat = t1 <= Real(0) ? 4 : (t1 >= Real(1) ? 6 : 3);
    return P1;
  }
  beta[0] = Real(1) - t0;
  beta[1] = t0;
  beta[2] = 0;
  *feat = f0;
  return P0;
}

// ------------------------------------------------------------ geometry pass
// Face normal of element e, computed from the marker positions.
template <class Real>
__device__ __forceinline__ V3<Real> face_normal(const IBArgs<Real>& a, int e) {
  if (a.NV == 2) {
    int p = a.E[2 * e], q = a.E[2 * e + 1];
    Real tx = node_dx(a, q, p, 0), tz = node_dx(a, q, p, 2);
    Real l = sqrt(tx * tx + tz * tz);
    return mk<Real>(tz / l, Real(0), -tx / l);
  }
  int p = a.E[3 * e], q = a.E[3 * e + 1], r = a.E[3 * e + 2];
  V3<Real> b = node_dv(a, q, p);
  V3<Real> c = node_dv(a, r, p);
  V3<Real> cr = cross(b, c);
  return (Real(1) / sqrt(dot(cr, cr))) * cr;
}

// One launch for the geometry of the step: threads [0, ne) store the unit
// outward face normals; threads [ne, ne + nn) store the vertex
// pseudo-normals, the angle-weighted sum of the incident face normals
// (Baerentzen and Aanaes 2005; in 2D the sum of the two segment normals),
// computing those normals themselves.
template <class Real>
__device__ __forceinline__ void geometry_body(const IBArgs<Real>& a, const Blk& blk) {
  int t = blk.x * blockDim.x + threadIdx.x;
  if (t < a.ne) {
    V3<Real> n = face_normal(a, t);
    a.en[3 * t] = n.x;
    a.en[3 * t + 1] = n.y;
    a.en[3 * t + 2] = n.z;
    const int* Et = a.E + a.NV * t;
    Real rv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int d = 0; d < 3; ++d) {
      const int o = a.xo[3 * Et[0] + d];
      a.eorg[3 * t + d] = o;
      for (int q = 0; q < a.NV; ++q) {
        rv[q][d] = node_off(a, Et[q], d, o);
        a.erel[3 * (a.NV * t + q) + d] = rv[q][d];
      }
    }
    // edge constants of the band's closest-point search (a segment keeps
    // ac = bc = 0)
    const V3<Real> A = mk<Real>(rv[0][0], rv[0][1], rv[0][2]), Bv = mk<Real>(rv[1][0], rv[1][1], rv[1][2]);
    const V3<Real> Cv = a.NV == 3 ? mk<Real>(rv[2][0], rv[2][1], rv[2][2]) : A;
    const V3<Real> ab = Bv - A, ac = a.NV == 3 ? Cv - A : mk<Real>(0, 0, 0), bc = a.NV == 3 ? Cv - Bv : mk<Real>(0, 0, 0);
    const Real d00 = dot(ab, ab), d01 = dot(ab, ac), d11 = dot(ac, ac), dbc = dot(bc, bc);
    const Real den = d00 * d11 - d01 * d01;
    Real* k = a.ecst + 16 * t;
    const Real kv[16] = {ab.x, ab.y, ab.z, ac.x, ac.y, ac.z, bc.x, bc.y, bc.z, d00, d01, d11,
                         d00 > Real(0) ? rcp_rn(d00) : Real(0), d11 > Real(0) ? rcp_rn(d11) : Real(0),
                         dbc > Real(0) ? rcp_rn(dbc) : Real(0), den > Real(0) ? rcp_rn(den) : Real(0)};
    for (int q = 0; q < 16; ++q) k[q] = kv[q];
    return;
  }
  int k = t - a.ne;
  if (k >= a.nn) return;
  V3<Real> s = mk<Real>(0, 0, 0);
  for (int j = a.inc_off[k]; j < a.inc_off[k + 1]; ++j) {
    int e = a.inc[j];
    V3<Real> n = face_normal(a, e);
    Real wgt = 1;
    if (a.NV == 3) {
      int q0 = a.E[3 * e], q1 = a.E[3 * e + 1], q2 = a.E[3 * e + 2];
      int u = q0 == k ? q1 : (q1 == k ? q2 : q0);
      int v = q0 == k ? q2 : (q1 == k ? q0 : q1);
      V3<Real> eu = node_dv(a, u, k);
      V3<Real> ev = node_dv(a, v, k);
      Real c = dot(eu, ev) / sqrt(dot(eu, eu) * dot(ev, ev));
      wgt = acos(fmin(Real(1), fmax(Real(-1), c)));
    }
    s = s + wgt * n;
  }
  a.vn[3 * k] = s.x;
  a.vn[3 * k + 1] = s.y;
  a.vn[3 * k + 2] = s.z;
}
template <class Real>
__global__ void k_geometry(const __grid_constant__ IBArgs<Real> a, int snap) {
  // start-of-step bookkeeping of the single-lattice path: clear the
  // coupling sums and, with snap, take the snapshot of the marker box and
  // reset its accumulator
  const long long n3 = 3ll * a.nn;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    a.ncpl[i] = 0;
  if (snap && blockIdx.x == 0 && threadIdx.x < 6) {
    a.box[6 + threadIdx.x] = a.box[threadIdx.x];
    a.box[threadIdx.x] = 0x7F7F7F7F;
  }
  geometry_body(a, hw_blk());
}

// Marker bounding box.  The advection kernel accumulates floor(min X) and
// -ceil(max X) per axis with integer atomicMin into box[0..5] (reset to a
// large value after use); k_box does the same from scratch at set-up, and
// both store the split X = xo + xr of the positions.
template <class Real>
__device__ __forceinline__ void box_body(const IBArgs<Real>& a, const Blk& blk) {
  int k = blk.x * blockDim.x + threadIdx.x;
  if (k >= a.nn) return;
  for (int d = 0; d < 3; ++d) {
    double v = fmax(-1e8, fmin(1e8, a.X[3 * k + d]));
    atomicMin(a.box + d, (int)floor(v));
    atomicMin(a.box + 3 + d, -(int)ceil(v));
    split_coord(a.X[3 * k + d], a.xo + 3 * k + d, a.xr + 3 * k + d);
  }
}
template <class Real>
__global__ void k_box(const __grid_constant__ IBArgs<Real> a) {
  box_body(a, hw_blk());
}

// The box of cells the profile visits: the step's marker box widened by
// dc + 2 cells (unwrapped; walls clamp z; at most one period per axis).
template <class Real>
__device__ __forceinline__ void profile_box(const IBArgs<Real>& a, int* lo, int* hi) {
  marker_box(a.boxc, (int)ceil(a.dc) + 2, a.G, a.dim == 2, lo, hi);
}

// Wrap a coordinate into [0, n): a compare and add within one period of the
// range, the division beyond it.
__device__ __forceinline__ int wrap_coord(int v, int n) {
  if (v < 0) v += n;
  else if (v >= n) v -= n;
  if ((unsigned)v >= (unsigned)n) {
    v %= n;
    if (v < 0) v += n;
  }
  return v;
}

template <class Real>
__device__ __forceinline__ long long cell_of(const IBArgs<Real>& a, const int* pc) {
  if (a.G.wall && (pc[2] < 0 || pc[2] >= a.G.nz)) return -1;
  const int x = wrap_coord(pc[0], a.G.nx), y = wrap_coord(pc[1], a.G.ny), z = wrap_coord(pc[2], a.G.nz);
  return ((long long)z * a.G.ny + y) * a.G.nx + x;
}

// Fixed-point conversions from the bits of an FP32 value, equal to the
// conversions of the exactly scaled number (v * 2^s) that the FP64 path
// makes, without FP64 arithmetic (a slow pipe on this GPU).
// floor(v 2^s) for finite v >= 0, v 2^s < 2^63:
__device__ __forceinline__ unsigned long long scaled_floor_u64(float v, int s) {
  const unsigned b = __float_as_uint(v);
  int e = (int)((b >> 23) & 0xFFu);
  unsigned long long m = b & 0x7FFFFFu;
  if (e) m |= 0x800000u;
  else e = 1;
  const int sh = e - 150 + s;  // v = m 2^(e - 150)
  return sh >= 0 ? m << sh : (sh > -24 ? m >> -sh : 0ull);
}
// rint(v 2^s), ties to even; saturates at +-2^62:
__device__ __forceinline__ long long scaled_rint_s64(float v, int s) {
  const unsigned b = __float_as_uint(v);
  int e = (int)((b >> 23) & 0xFFu);
  unsigned long long m = b & 0x7FFFFFu;
  if (e) m |= 0x800000u;
  else e = 1;
  const int sh = e - 150 + s;
  unsigned long long r;
  if (sh >= 0) {
    r = sh <= 38 ? m << sh : (1ull << 62);
  } else if (sh >= -24) {
    const int k = -sh;
    const unsigned long long q = m >> k, rem = m - (q << k), half = 1ull << (k - 1);
    r = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  } else {
    r = 0;
  }
  return (b >> 31) ? -(long long)r : (long long)r;
}
// distance part of a scatter key: the distance on a grid of 2^-34
__device__ __forceinline__ unsigned long long dist_code(float d) { return scaled_floor_u64(d, 34); }
__device__ __forceinline__ unsigned long long dist_code(double d) {
  return (unsigned long long)(d * 17179869184.0);
}

// Squared distance from a point to a triangle (or a segment), without
// branches: the projection onto the plane when it falls inside the
// triangle, else the nearest of the three clamped edge projections.  The
// per-face quantities are set up once; a point costs about fifty
// arithmetic instructions and no divergence.
template <class Real>
struct FaceDist {
  V3<Real> A, B, ab, ac, bc;
  Real d00, d01, d11, i00, i11, ibc, iden;
  bool tri;
  static constexpr int NC = 22;  // constants kept in shared memory
  static constexpr int NCP = 24; // row stride of the shared copy (16-byte rows for FP32)
  __device__ __forceinline__ FaceDist() {}
  __device__ __forceinline__ void store(Real* p) const {
    const Real v[NC] = {A.x,  A.y,  A.z,  B.x,  B.y,  B.z,  ab.x, ab.y, ab.z, ac.x, ac.y,
                        ac.z, bc.x, bc.y, bc.z, d00,  d01,  d11,  i00,  i11,  ibc,  iden};
    for (int i = 0; i < NC; ++i) p[i] = v[i];
  }
  __device__ __forceinline__ static FaceDist load(const Real* p, bool is_tri) {
    if constexpr (sizeof(Real) == 4) {  // six 16-byte loads of the padded row
      float v[NCP];
#pragma unroll
      for (int i = 0; i < NCP / 4; ++i) {
        const float4 q = reinterpret_cast<const float4*>(p)[i];
        v[4 * i] = q.x;
        v[4 * i + 1] = q.y;
        v[4 * i + 2] = q.z;
        v[4 * i + 3] = q.w;
      }
      FaceDist f;
      f.A = mk<Real>(v[0], v[1], v[2]);
      f.B = mk<Real>(v[3], v[4], v[5]);
      f.ab = mk<Real>(v[6], v[7], v[8]);
      f.ac = mk<Real>(v[9], v[10], v[11]);
      f.bc = mk<Real>(v[12], v[13], v[14]);
      f.d00 = v[15];
      f.d01 = v[16];
      f.d11 = v[17];
      f.i00 = v[18];
      f.i11 = v[19];
      f.ibc = v[20];
      f.iden = v[21];
      f.tri = is_tri;
      return f;
    }
    FaceDist f;
    f.A = mk<Real>(p[0], p[1], p[2]);
    f.B = mk<Real>(p[3], p[4], p[5]);
    f.ab = mk<Real>(p[6], p[7], p[8]);
    f.ac = mk<Real>(p[9], p[10], p[11]);
    f.bc = mk<Real>(p[12], p[13], p[14]);
    f.d00 = p[15];
    f.d01 = p[16];
    f.d11 = p[17];
    f.i00 = p[18];
    f.i11 = p[19];
    f.ibc = p[20];
    f.iden = p[21];
    f.tri = is_tri;
    return f;
  }
  __device__ __forceinline__ FaceDist(V3<Real> a, V3<Real> b, V3<Real> c, bool is_tri) : A(a), B(b), tri(is_tri) {
    ab = b - a;
    ac = c - a;
    bc = c - b;
    d00 = dot(ab, ab);
    d01 = dot(ab, ac);
    d11 = dot(ac, ac);
    const Real dbc = dot(bc, bc), den = d00 * d11 - d01 * d01;
    i00 = d00 > Real(0) ? rcp_rn(d00) : Real(0);  // degenerate edge: its first end
    i11 = d11 > Real(0) ? rcp_rn(d11) : Real(0);
    ibc = dbc > Real(0) ? rcp_rn(dbc) : Real(0);
    iden = den > Real(0) ? rcp_rn(den) : Real(0);  // degenerate face: edges only
  }
  __device__ __forceinline__ Real dist2(V3<Real> x) const {
    const V3<Real> ap = x - A;
    const Real d20 = dot(ap, ab);
    const Real t0 = fmin(Real(1), fmax(Real(0), d20 * i00));
    const V3<Real> e0 = ap - t0 * ab;
    Real best = dot(e0, e0);
    if (!tri) return best;
    const Real d21 = dot(ap, ac);
    const Real t1 = fmin(Real(1), fmax(Real(0), d21 * i11));
    const V3<Real> e1 = ap - t1 * ac;
    const V3<Real> bp = x - B;
    const Real t2 = fmin(Real(1), fmax(Real(0), dot(bp, bc) * ibc));
    const V3<Real> e2 = bp - t2 * bc;
    best = fmin(best, fmin(dot(e1, e1), dot(e2, e2)));
    const Real v = (d11 * d20 - d01 * d21) * iden, w = (d00 * d21 - d01 * d20) * iden;
    const V3<Real> q = ap - v * ab - w * ac;
    const bool inside = iden > Real(0) && v >= Real(0) && w >= Real(0) && v + w <= Real(1);
    return inside ? dot(q, q) : best;
  }
};

// ------------------------------------------------------------ distance scatter
// Every cell within dc of the membrane must receive the key (distance,
// element) of its nearest element; keys are combined with atomicMin.  The
// nearest point P of a cell x lies in the interior of a face, in the
// interior of an edge or on a vertex, and x - P lies in the normal cone of
// that feature: the face normal, the wedge of the two face normals of an
// edge, the cone of the face normals around a vertex (in 2D: segment normal,
// and the fan of the two segment normals at a marker).  Each feature sweeps
// the cells x = P + t m, P on the feature, m in its cone (either sign),
// |t| < dc, and offers every cell the exact distance to the faces that
// contain the feature.  The sweep runs slice by slice along an axis k in
// which all cone generators have a component of one sign; on slice x_k = c
// the region lies in the convex hull of the points where the rays from the
// feature's corners along the generators meet the slice, whose bounding box
// is enumerated.  Distances are compared on a grid of 2^-34 lattice units,
// ties going to the lowest element index.
constexpr int MAXG = 12;  // generators (and faces) per feature
constexpr int SCAT_W = 4;       // slices per lane per round
constexpr int SCAT_SPLIT = 4;   // warps sharing one group of 32 features (round r goes to r % SCAT_SPLIT)
// warps per block (every lane sweeps one feature): FP64 halves them to keep
// the shared memory under the static limit
template <class Real> constexpr int scatter_warps() { return sizeof(Real) == 4 ? 4 : 2; }

// Shared memory of one warp: lane l's feature in row l.
template <class Real>
struct ScatterWarp {
  Real cb[32][9];               // corners relative to the feature's origin
  Real gk[32][MAXG];            // 1 / generator component along the slice axis
  Real ga[32][MAXG];            // generator components along the two other axes
  Real gb[32][MAXG];
  alignas(16) Real fd[32][FaceDist<Real>::NCP];  // distance constants of the offered face
  int4 sl[32][SCAT_W];          // the round's slices: a0, b0, width, cumulative cells
  int4 ft[32][2];               // origin cell (wrapped) and packed axes; face, first slice
};

// One lane per feature, geometry in Real relative to an integer origin (the
// lattice cell below the first corner), so the FP32 build sweeps in single
// precision without losing accuracy; slice boxes are widened by 1e-3 cells
// to stay conservative under rounding.  The warp then shares out the cells:
// per round every lane sizes SCAT_W slices of its feature, a warp prefix sum
// lays all their cells end to end, and the lanes take them round-robin.
// SCAT_SPLIT virtual blocks set up the same features and take turns over
// the rounds (the set-up is short; the rounds are not).
// A feature offers only its lowest-index face: if the nearest point P of a
// cell lies on the feature, every face containing the feature is at exactly
// |x - P|, so that face carries the key the tie rule selects; faces offered
// for cells whose nearest point lies elsewhere are at their exact (larger or
// equal) distance and cannot win wrongly.
template <class Real>
__device__ __forceinline__ void dist_scatter_body(const IBArgs<Real>& a, const Blk& blk) {
  constexpr int SW = scatter_warps<Real>();
  __shared__ ScatterWarp<Real> smw[SW];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= SW) return;
  ScatterWarp<Real>& sm = smw[w];
  const int nfeat = a.ne + (a.NV == 3 ? a.nedge : 0) + a.nn;
  const int grp = blk.x / SCAT_SPLIT, phase = blk.x % SCAT_SPLIT;
  const int f = (grp * SW + w) * 32 + lane;
  if (__ballot_sync(0xffffffffu, f < nfeat) == 0) return;
  // ---- the lane's feature: corners, cone generators (the normals of the
  // faces containing it), slice axis and range, offered face
  int kind = 0, nB = 0, nG = 0, i0 = 0, corners[3] = {0, 0, 0};
  if (f < nfeat) {
    if (f < a.ne) {  // face (3D) or segment (2D)
      nB = a.NV;
      nG = 1;
      for (int q = 0; q < a.NV; ++q) corners[q] = a.E[a.NV * f + q];
    } else if (a.NV == 3 && f < a.ne + a.nedge) {  // edge
      kind = 1;
      const int* ed = a.edges + 4 * (f - a.ne);
      corners[0] = ed[0];
      corners[1] = ed[1];
      nB = 2;
      nG = 2;
    } else {  // vertex
      kind = 2;
      const int v = f - a.ne - (a.NV == 3 ? a.nedge : 0);
      corners[0] = v;
      nB = 1;
      i0 = a.inc_off[v];
      nG = min(a.inc_off[v + 1] - i0, MAXG);
    }
  }
  auto face_of = [&](int j) { return kind == 0 ? f : (kind == 1 ? a.edges[4 * (f - a.ne) + 2 + j] : a.inc[i0 + j]); };
  bool ok = nG > 0;
  int o[3] = {0, 0, 0}, tmin = 0x7fffffff;
  Real S[3] = {0, 0, 0};
  if (ok) {
    for (int d = 0; d < 3; ++d) o[d] = a.xo[3 * corners[0] + d];
    if (a.dim == 2) o[1] = 0;
    for (int j = 0; j < nG; ++j) {
      const int t = face_of(j);
      tmin = min(tmin, t);
      for (int d = 0; d < 3; ++d) {
        const Real g = a.en[3 * t + d];
        S[d] += g;
        ok &= fabs(g) <= Real(1.001);
      }
    }
    for (int q = 0; q < nB; ++q)
      for (int d = 0; d < 3; ++d) {
        const Real b = node_off(a, corners[q], d, o[d]);
        sm.cb[lane][3 * q + d] = b;
        ok &= fabs(b) < Real(1e6);  // rejects NaN/Inf
      }
    if (!ok) atomicOr(a.status, (unsigned)ST_NAN);
  }
  // slice axis: largest component of the generator sum, all generators of one sign
  int k = 0;
  if (a.dim == 3) {
    if (fabs(S[1]) > fabs(S[k])) k = 1;
    if (fabs(S[2]) > fabs(S[k])) k = 2;
  } else {
    k = fabs(S[2]) > fabs(S[0]) ? 2 : 0;
  }
  int oa, ob;
  if (a.dim == 3) { oa = k == 0 ? 1 : 0; ob = k == 2 ? 1 : 2; }
  else { oa = k == 0 ? 2 : 0; ob = 1; }
  const Real dc = a.dc, eps = Real(1e-3);
  int c0 = 0, nsl = 0;
  bool wide = false;
  if (ok) {
    Real gmin = Real(1e30f);
    for (int j = 0; j < nG; ++j) {
      const int t = face_of(j);
      const Real gkj = a.en[3 * t + k];
      gmin = fmin(gmin, gkj * (S[k] >= 0 ? Real(1) : Real(-1)));
      // (the rectangles are widened by eps, far above the rounding of a product)
      sm.gk[lane][j] = rcp_rn(gkj);
      sm.ga[lane][j] = a.en[3 * t + oa];
      sm.gb[lane][j] = a.en[3 * t + ob];
    }
    wide = gmin < Real(0.25);  // a generator nearly parallel to the slices
    Real bmin = 1e30f, bmax = -1e30f;
    for (int q = 0; q < nB; ++q) {
      bmin = fmin(bmin, sm.cb[lane][3 * q + k]);
      bmax = fmax(bmax, sm.cb[lane][3 * q + k]);
    }
    c0 = (int)ceil(bmin - dc - eps);
    nsl = (int)floor(bmax + dc + eps) - c0 + 1;
    V3<Real> vq[3];
    for (int q = 0; q < 3; ++q) {
      const int m = a.E[a.NV * tmin + min(q, a.NV - 1)];
      vq[q] = mk<Real>(node_off(a, m, 0, o[0]), node_off(a, m, 1, o[1]), node_off(a, m, 2, o[2]));
    }
    FaceDist<Real>(vq[0], vq[1], vq[2], a.NV == 3).store(sm.fd[lane]);
    const int ow[3] = {wrap_coord(o[0], a.G.nx), wrap_coord(o[1], a.G.ny), a.G.wall ? o[2] : wrap_coord(o[2], a.G.nz)};
    sm.ft[lane][0] = make_int4(ow[0], ow[1], ow[2], k | (oa << 2) | (ob << 4));
    sm.ft[lane][1] = make_int4(tmin, c0, 0, 0);
  }
  // bounding rectangle of the cone's cross-section in slice c: origin (a0,
  // b0), width wa, cnt cells (0 when empty or flagged as too wide)
  auto slice_rect = [&](int c, int& a0, int& b0, int& wa, int& cnt) {
    Real lo0 = 1e30f, hi0 = -1e30f, lo1 = 1e30f, hi1 = -1e30f;
    for (int q = 0; q < nB; ++q) {
      const Real bk = sm.cb[lane][3 * q + k], ba = sm.cb[lane][3 * q + oa], bb = sm.cb[lane][3 * q + ob];
      if (!wide) {
        for (int j = 0; j < nG; ++j) {
          const Real t = ((Real)c - bk) * sm.gk[lane][j];
          const Real pa = ba + t * sm.ga[lane][j], pb = bb + t * sm.gb[lane][j];
          lo0 = fmin(lo0, pa); hi0 = fmax(hi0, pa);
          lo1 = fmin(lo1, pb); hi1 = fmax(hi1, pb);
        }
      } else {  // conservative: the feature's box widened by dc
        lo0 = fmin(lo0, ba - dc); hi0 = fmax(hi0, ba + dc);
        lo1 = fmin(lo1, bb - dc); hi1 = fmax(hi1, bb + dc);
      }
    }
    a0 = (int)ceil(lo0 - eps);
    const int a1 = (int)floor(hi0 + eps);
    int b1 = 0;
    b0 = 0;
    if (a.dim == 3) { b0 = (int)ceil(lo1 - eps); b1 = (int)floor(hi1 + eps); }
    const int wb = b1 - b0 + 1;
    wa = a1 - a0 + 1;
    cnt = 0;
    if (wa > 0 && wb > 0) {
      if (wa > 1024 || wb > 1024) atomicOr(a.status, (unsigned)ST_OVERFLOW);  // bounded work, flagged
      else cnt = wa * wb;
    }
    if (cnt == 0) wa = 1;
  };
  const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)((nsl + SCAT_W - 1) / SCAT_W));
  const Real dc2 = dc * dc;
  for (int r = phase; r < rounds; r += SCAT_SPLIT) {
    int tot = 0;
#pragma unroll
    for (int h = 0; h < SCAT_W; ++h) {
      const int sidx = r * SCAT_W + h;
      int a0 = 0, b0 = 0, wa = 1, cnt = 0;
      if (sidx < nsl) slice_rect(c0 + sidx, a0, b0, wa, cnt);
      tot += cnt;
      sm.sl[lane][h] = make_int4(a0, b0, wa, tot);
    }
    int incl = tot;
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, sh);
      if (lane >= sh) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    for (int j0 = 0; j0 < total; j0 += 32) {
      const int i = j0 + lane;
      // lane holding cell i: the first lane whose inclusive prefix exceeds i
      int L = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, L + step - 1);
        if (v <= i) L += step;
      }
      const int base = __shfl_sync(0xffffffffu, incl, L) - __shfl_sync(0xffffffffu, tot, L);
      if (i >= total) continue;
      int jj = i - base;
      // its slice: the first whose cumulative count exceeds jj
      int4 e = sm.sl[L][0];
      int h = 0, prev = 0;
#pragma unroll
      for (int q = 1; q < SCAT_W; ++q) {
        if (jj >= e.w) {
          prev = e.w;
          e = sm.sl[L][q];
          h = q;
        }
      }
      jj -= prev;
      // jj / wa: jj < 2^20 and wa <= 1024 keep the product within 2^-13 of the
      // true (jj + 1/2) / wa, whose fraction is at least 2^-11 from an
      // integer, so the truncation is exact
      const int qb = (int)(((float)jj + 0.5f) * __frcp_rn((float)e.z));
      const int4 F0 = sm.ft[L][0], F1 = sm.ft[L][1];
      const int kk = F0.w & 3, ka = (F0.w >> 2) & 3, kb = (F0.w >> 4) & 3;
      int rr[3];
      rr[kk] = F1.y + r * SCAT_W + h;
      rr[ka] = e.x + (jj - qb * e.z);
      rr[kb] = a.dim == 3 ? e.y + qb : 0;
      const int pc[3] = {F0.x + rr[0], F0.y + rr[1], F0.z + rr[2]};
      const long long cell = cell_of(a, pc);
      if (cell < 0) continue;
      const Real d2 = FaceDist<Real>::load(sm.fd[L], a.NV == 3).dist2(mk<Real>((Real)rr[0], (Real)rr[1], (Real)rr[2]));
      if (!(d2 < dc2)) continue;
      const unsigned long long key = (dist_code(sqrt(d2)) << 24) | (unsigned long long)F1.x;
      atomicMin(a.key + cell, key);  // no return value: a fire-and-forget reduction
    }
    __syncwarp();  // the next round rewrites the slice table
  }
}
// Persistent over nvb virtual blocks (grid capped by the caller).
template <class Real>
__global__ void __launch_bounds__(scatter_warps<Real>() * 32) k_dist_scatter(const __grid_constant__ IBArgs<Real> a, int nvb) {
  for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) dist_scatter_body(a, Blk{vb, 0, 0, nvb, 1, 1});
}

// Sign of x - P relative to the membrane at the closest feature (interior:
// element normal; edge: sum of the two adjacent normals; vertex: vertex
// pseudo-normal): +1 inside (d > 0 in eq. Iprofile), -1 outside.
template <class Real>
__device__ __forceinline__ Real feature_sign(const IBArgs<Real>& a, int e, int feat, V3<Real> xmP) {
  V3<Real> N;
  if (feat == 0) {
    N = mk<Real>(a.en[3 * e], a.en[3 * e + 1], a.en[3 * e + 2]);
  } else if (a.NV == 3 && feat <= 3) {
    int f = a.adj[3 * e + (feat - 1)];
    N = mk<Real>(a.en[3 * e] + a.en[3 * f], a.en[3 * e + 1] + a.en[3 * f + 1], a.en[3 * e + 2] + a.en[3 * f + 2]);
  } else {
    int q = feat - 4;
    int k = a.E[a.NV * e + q];
    N = mk<Real>(a.vn[3 * k], a.vn[3 * k + 1], a.vn[3 * k + 2]);
  }
  // x - P points outward for a cell outside
  return dot(xmP, N) > Real(0) ? Real(-1) : Real(1);
}

// Fixed-point scale of the coupling sums: integer additions make the
// per-element totals independent of the order of the contributions.
#define CPL_SCALE 1125899906842624.0  // 2^50
__device__ __forceinline__ long long cpl_fixed(float v) { return scaled_rint_s64(v, 50); }
__device__ __forceinline__ long long cpl_fixed(double v) { return llrint(v * CPL_SCALE); }

// Band cells of the marker box (one thread per cell, x fastest): signed
// distance from the nearest element, I = (1 + tanh(d/(2 alpha)))/2 (eq.
// Iprofile), owner element, and the coupling force contributions (eq.
// DiscreteCF from eq. DiscreteCE): node k of the owner receives
//   kappa_c (psi - I) sech^2(d/(2 alpha))/(4 alpha) * (-s beta_k (x - P)/|x - P|),
// summed per marker in fixed point (lanes of a warp with the same element
// are combined before one atomic per node; a reduction per lane measured
// slower on the contended addresses).  Cells without a key are marked -1 for
// the column fill; keys are cleared for the next step.  A cell that was a
// band cell in the previous step and is not one now lies beyond dc on the
// side of its last distance (the membrane moves less than half a cell per
// step and cannot cross a cell farther than dc from it): it takes +-dc and
// I_in/I_out here, so that between fresh starts the column fill, which
// would find the same sides, is not needed.
template <class Real>
__device__ __forceinline__ void band_body(const IBArgs<Real>& a, const Blk& blk) {
  int blo[3], bhi[3];
  profile_box(a, blo, bhi);
  const int bx0 = blo[0], by0 = blo[1], bz0 = blo[2];
  const int wx = bhi[0] - bx0 + 1, wy = bhi[1] - by0 + 1, wz = bhi[2] - bz0 + 1;
  const long long total = (long long)wx * wy * wz;
  const bool full[3] = {wx == a.G.nx, a.dim == 3 && wy == a.G.ny, !a.G.wall && wz == a.G.nz};
  const Real al = a.alpha, Iin = a.Iin, Iout = a.Iout;
  // the box origin wrapped into the lattice: cells are indexed from it, the
  // geometry uses the unwrapped coordinates
  const int ox = wrap_coord(bx0, a.G.nx), oy = wrap_coord(by0, a.G.ny), oz = a.G.wall ? bz0 : wrap_coord(bz0, a.G.nz);
  const bool narrow = total <= 0xFFFFFFFFll;
  const long long stride = (long long)blk.gx * blockDim.x;
  for (long long t0 = (long long)blk.x * blockDim.x; t0 < total; t0 += stride) {
    const long long t = t0 + threadIdx.x;
    int e = -1;
    Real acc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (t < total) {
      int ix, iy, iz;
      if (narrow) {  // 32-bit division
        const unsigned tt = (unsigned)t, row = tt / (unsigned)wx, zz = row / (unsigned)wy;
        ix = (int)(tt - row * (unsigned)wx);
        iy = (int)(row - zz * (unsigned)wy);
        iz = (int)zz;
      } else {
        ix = (int)(t % wx);
        iy = (int)((t / wx) % wy);
        iz = (int)(t / ((long long)wx * wy));
      }
      const int pc[3] = {bx0 + ix, by0 + iy, bz0 + iz};
      const int pw[3] = {ox + ix, oy + iy, oz + iz};
      long long c = cell_of(a, pw);
      if (c >= 0) {
        // psi is requested with the key, so its latency overlaps the key's
        // and the element's (it is needed only for band cells)
        const Real psic = a.psi[c];
        unsigned long long key = a.key[c];
        if (key == KEY_NONE) {
          if (a.own[c] >= 0) {  // left the band since the previous step
            const bool in = a.dsel[c] > Real(0);
            a.dsel[c] = in ? a.dc : -a.dc;
            a.I[c] = in ? Iin : Iout;
          }
          a.own[c] = -1;
        } else {
          e = (int)(key & 0xFFFFFF);
          a.key[c] = KEY_NONE;
          Real beta[3];
          int feat;
          // Along an axis where the box spans a whole period a band cell may
          // sit one period away from the element that keyed it: measure from
          // the image of the cell nearest to the element (unique, as
          // periodic sides are at least 2 dc + 8).  A box narrower than the
          // period holds every band cell at that image already.
          // (the element origin, floor of its first vertex, is within a cell
          // of it: the nearest image is the same)
          int pi[3] = {pc[0], pc[1], pc[2]};
          if (full[0] | full[1] | full[2]) {
            const int* eo = a.eorg + 3 * e;
            if (full[0]) pi[0] += a.G.nx * __float2int_rn((float)(eo[0] - pi[0]) / (float)a.G.nx);
            if (full[1]) pi[1] += a.G.ny * __float2int_rn((float)(eo[1] - pi[1]) / (float)a.G.ny);
            if (full[2]) pi[2] += a.G.nz * __float2int_rn((float)(eo[2] - pi[2]) / (float)a.G.nz);
          }
          V3<Real> P = elem_closest(a, e, pi, beta, &feat);
          V3<Real> xmP = mk<Real>(-P.x, -P.y, -P.z);
          Real dist = sqrt(dot(xmP, xmP));
          Real s = feature_sign(a, e, feat, xmP);
          Real d = s * dist;
          Real I = Real(0.5) * (Real(1) + tanh(d / (Real(2) * al)));
          a.dsel[c] = d;
          a.own[c] = e;
          a.I[c] = I;
          Real ch = cosh(d / (Real(2) * al));
          Real coef = a.kc * (psic - I) / (ch * ch) / (Real(4) * al);
          V3<Real> dir;
          if (dist > Real(1e-12)) dir = (-s / dist) * xmP;
          else dir = mk<Real>(a.en[3 * e], a.en[3 * e + 1], a.en[3 * e + 2]);
#pragma unroll
          for (int q = 0; q < 3; ++q) {  // beta[2] = 0 for segments
            acc[q][0] = coef * beta[q] * dir.x;
            acc[q][1] = coef * beta[q] * dir.y;
            acc[q][2] = coef * beta[q] * dir.z;
          }
        }
      }
    }
    // combine lanes that share an element, one fixed-point atomic per group
    const unsigned active = __ballot_sync(0xffffffffu, e >= 0);
    if (e >= 0) {
      const unsigned grp = __match_any_sync(active, e);
      const int leader = __ffs(grp) - 1;
      const int lane = threadIdx.x & 31;
      long long v[9], sum[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        v[i] = cpl_fixed(acc[i / 3][i % 3]);
        sum[i] = 0;
      }
      // sum over the group (integers: any order gives the same total)
      for (unsigned m = grp; m; m &= m - 1) {
        const int src = __ffs(m) - 1;
#pragma unroll
        for (int i = 0; i < 9; ++i) sum[i] += __shfl_sync(grp, v[i], src);
      }
      if (lane == leader) {  // straight to the element's nodes
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (q >= a.NV) break;
          const int node = a.E[a.NV * e + q];
#pragma unroll
          for (int d = 0; d < 3; ++d)
            if (sum[3 * q + d] != 0) atomicAdd(a.ncpl + 3 * node + d, (unsigned long long)sum[3 * q + d]);
        }
      }
    }
  }
}
template <class Real>
__global__ void k_band(const __grid_constant__ IBArgs<Real> a) {
  band_body(a, hw_blk());
}

// Cells of the box farther than dc from the membrane: one warp per column
// along z, 32 cells at a time.  A cell outside the band takes the side of
// the nearest band cell below it (the membrane cannot be crossed between two
// cells that are both farther than dc from it; the bottom of the box is
// outside every capsule): d = +dc inside, -dc outside.
template <class Real>
__device__ __forceinline__ void fill_body(const IBArgs<Real>& a, const Blk& blk) {
  int blo[3], bhi[3];
  profile_box(a, blo, bhi);
  const int bx0 = blo[0], by0 = blo[1], bz0 = blo[2];
  const int wx = bhi[0] - bx0 + 1, wy = bhi[1] - by0 + 1, wz = bhi[2] - bz0 + 1;
  const int col = (blk.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (col >= wx * wy) return;
  const Real dc = a.dc, Iin = a.Iin, Iout = a.Iout;
  const Geo& G = a.G;
  const long long colc = (long long)wrap_coord(by0 + col / wx, G.ny) * G.nx + wrap_coord(bx0 + col % wx, G.nx);
  const long long plane = (long long)G.nx * G.ny;
  bool inside = false;  // status carried from the chunk below
  for (int z0 = 0; z0 < wz; z0 += 128) {
    // the loads of up to four chunks of 32 cells first (dsel is read for
    // every cell, used for band cells only), then the scans
    long long cq[4];
    int ownq[4];
    Real dq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int z = z0 + 32 * q + lane, pz = bz0 + z;
      cq[q] = -1;
      ownq[q] = -1;
      dq[q] = 0;
      if (z < wz && (!G.wall || (pz >= 0 && pz < G.nz))) {
        cq[q] = (long long)(G.wall ? pz : wrap_coord(pz, G.nz)) * plane + colc;
        ownq[q] = a.own[cq[q]];
        dq[q] = a.dsel[cq[q]];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (z0 + 32 * q >= wz) break;
      const long long c = cq[q];
      const bool band = c >= 0 && ownq[q] >= 0, sgn = band && dq[q] > Real(0);
      const unsigned bm = __ballot_sync(0xffffffffu, band);
      const unsigned sm = __ballot_sync(0xffffffffu, sgn);
      const unsigned below = bm & ((1u << lane) - 1u);
      const bool my = below ? ((sm >> (31 - __clz(below))) & 1u) : inside;
      if (c >= 0 && !band) {
        a.dsel[c] = my ? dc : -dc;
        a.I[c] = my ? Iin : Iout;
      }
      // carry: the status at the top band cell of the chunk
      inside = bm ? ((sm >> (31 - __clz(bm))) & 1u) : inside;
    }
  }
}
template <class Real>
__global__ void k_fill(const __grid_constant__ IBArgs<Real> a) {
  fill_body(a, hw_blk());
}

// ------------------------------------------------------------ elastic forces
constexpr int NODEF_WARPS = 4;  // warps per block of the node-force kernel (at most)

// Forward-mode dual number with derivatives with respect to one node.
template <class T>
struct D3 {
  T v, d0, d1, d2;
};
template <class T> TLB_HD D3<T> dc(T v) { return {v, 0, 0, 0}; }
template <class T> TLB_HD D3<T> operator+(D3<T> a, D3<T> b) { return {a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2}; }
template <class T> TLB_HD D3<T> operator-(D3<T> a, D3<T> b) { return {a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2}; }
template <class T> TLB_HD D3<T> operator*(D3<T> a, D3<T> b) {
  return {a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2};
}
template <class T> TLB_HD D3<T> operator*(T s, D3<T> a) { return {s * a.v, s * a.d0, s * a.d1, s * a.d2}; }
template <class T> TLB_HD D3<T> operator/(D3<T> a, D3<T> b) {
  T ib = T(1) / b.v;
  T q = a.v * ib;
  return {q, (a.d0 - q * b.d0) * ib, (a.d1 - q * b.d1) * ib, (a.d2 - q * b.d2) * ib};
}
template <class T> TLB_HD D3<T> dsqrt(D3<T> a) {
  T s = sqrt(a.v);
  T h = T(0.5) / s;
  return {s, a.d0 * h, a.d1 * h, a.d2 * h};
}
template <class T> using DV = V3<D3<T>>;
template <class T> TLB_HD DV<T> dsub(DV<T> a, DV<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> TLB_HD D3<T> ddot(DV<T> a, DV<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> TLB_HD DV<T> dcross(DV<T> a, DV<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Position of node j relative to the seed node k, differentiated with
// respect to X_k (the seed carries derivative -1 in every other node's frame:
// we place the origin at X_k so only the seed itself moves).
template <class Real>
__device__ __forceinline__ DV<Real> dnode(const IBArgs<Real>& a, int j, int k) {
  DV<Real> r;
  r.x = dc<Real>(node_dx(a, j, k, 0));
  r.y = dc<Real>(node_dx(a, j, k, 1));
  r.z = dc<Real>(node_dx(a, j, k, 2));
  if (j == k) { r.x.d0 = 1; r.y.d1 = 1; r.z.d2 = 1; }
  return r;
}

// Skalak energy of triangle t (shear modulus G, area ratio C):
// W = (G/4)(I1^2 + 2 I1 - 2 I2 + C I2^2), I1 = tr(G0^-1 g) - 2, I2 = det(G0^-1 g) - 1.
template <class Real>
__device__ __forceinline__ D3<Real> skalak_dual(const IBArgs<Real>& a, int t, int k) {
  int p = a.E[3 * t], q = a.E[3 * t + 1], r = a.E[3 * t + 2];
  DV<Real> xp = dnode(a, p, k), xq = dnode(a, q, k), xr = dnode(a, r, k);
  DV<Real> e1 = dsub(xq, xp), e2 = dsub(xr, xp);
  D3<Real> g11 = ddot(e1, e1), g12 = ddot(e1, e2), g22 = ddot(e2, e2);
  const Real* K = a.skc + 5 * t;
  D3<Real> tr = K[0] * g11 + K[1] * g12 + K[2] * g22;
  D3<Real> det = K[3] * (g11 * g22 - g12 * g12);
  D3<Real> I1 = tr - dc<Real>(2), I2 = det - dc<Real>(1);
  int cap = a.ecap[t];
  Real G = a.capr[2 * a.ncaps + cap], C = a.capr[3 * a.ncaps + cap];
  D3<Real> w = (G * Real(0.25)) * (I1 * I1 + Real(2) * I1 - Real(2) * I2 + C * (I2 * I2));
  return K[4] * w;
}

// Helfrich energy of vertex v: kb |sum_T (cot_k (x_v - x_j) + cot_j (x_v - x_k))|^2 / (8 A_v)
// with A_v the mixed Voronoi area (Meyer et al. 2003).  One term: the
// contributions of face t of v to the sums K and A, differentiated with
// respect to X_k.
template <class Real>
__device__ __forceinline__ void helfrich_term(const IBArgs<Real>& a, int v, int t, int k, DV<Real>& Kc, D3<Real>& Ac) {
  int q0 = a.E[3 * t], q1 = a.E[3 * t + 1], q2 = a.E[3 * t + 2];
  int j = q0 == v ? q1 : (q1 == v ? q2 : q0);
  int kk = q0 == v ? q2 : (q1 == v ? q0 : q1);
  DV<Real> xv = dnode(a, v, k), xj = dnode(a, j, k), xk = dnode(a, kk, k);
  DV<Real> vj = dsub(xv, xj), vk = dsub(xv, xk);
  DV<Real> kj = dsub(xk, xj), jk = dsub(xj, xk);
  DV<Real> c1 = dcross(vj, kj), c2 = dcross(vk, jk);
  D3<Real> cotj = ddot(vj, kj) / dsqrt(ddot(c1, c1));
  D3<Real> cotk = ddot(vk, jk) / dsqrt(ddot(c2, c2));
  Kc.x = cotk * vj.x + cotj * vk.x;
  Kc.y = cotk * vj.y + cotj * vk.y;
  Kc.z = cotk * vj.z + cotj * vk.z;
  DV<Real> ej = dsub(xj, xv), ek = dsub(xk, xv);
  DV<Real> cr = dcross(ej, ek);
  D3<Real> area = Real(0.5) * dsqrt(ddot(cr, cr));
  Real dv = ddot(ej, ek).v, dj = ddot(vj, kj).v, dk = ddot(vk, jk).v;
  if (dv < 0) Ac = Real(0.5) * area;
  else if (dj < 0 || dk < 0) Ac = Real(0.25) * area;
  else Ac = Real(0.125) * (ddot(vj, vj) * cotk + ddot(vk, vk) * cotj);
}

// Elastic node forces, one warp per marker (2D stretching + bending; 3D
// Skalak + Helfrich, differentiated with forward-mode duals with respect to
// the marker).  In 3D lane t takes the Skalak term of incident face t, and
// the Helfrich terms of the marker and its 1-ring vertices are shared out
// as (vertex, face) pairs, 32 at a time: each lane stages its pair's
// contributions to K and A, the lane of each vertex adds them in face order
// and forms the vertex's energy.  Lane sums are combined by a fixed shuffle
// tree.  They depend on the marker positions only; the coupling force joins
// them in k_spread.
template <class Real>
__device__ __forceinline__ void node_forces_body(const IBArgs<Real>& a, const Blk& blk) {
  __shared__ Real hstage[NODEF_WARPS][32 * 16];  // one chunk of Helfrich pairs per warp
  const int k = (blk.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= a.nn) return;
  Real F[3] = {0, 0, 0};
  if (a.NV == 2) {
    if (lane == 0) {
      // 2D ring: segment l joins node l -> next(l) (eq. DiscreteSE), bending
      // at nodes prev, k, next (eqs. DiscreteBE, DiscreteTheta, DiscreteArcLength).
      const int cap = a.ncap[k];
      const Real ks = a.capr[cap], kb = a.capr[a.ncaps + cap];
      for (int side = 0; side < 2; ++side) {
        int e = a.inc[a.inc_off[k] + side];
        int p = a.E[2 * e], q = a.E[2 * e + 1];
        Real tx = node_dx(a, q, p, 0), tz = node_dx(a, q, p, 2);
        Real L = sqrt(tx * tx + tz * tz);
        Real T = ks * (L / (Real)a.ds0[e] - Real(1)) / L;
        Real sgn = (p == k) ? Real(1) : Real(-1);  // -dE/dX_p = +T t ; -dE/dX_q = -T t
        F[0] += sgn * T * tx;
        F[2] += sgn * T * tz;
      }
      int ms[3] = {a.rprev[k], k, a.rnext[k]};
      for (int mi = 0; mi < 3; ++mi) {
        int m = ms[mi], mp = a.rnext[m], mq = a.rprev[m];
        Real ax = node_dx(a, mp, m, 0), az = node_dx(a, mp, m, 2);
        Real bx = node_dx(a, m, mq, 0), bz = node_dx(a, m, mq, 2);
        Real la = sqrt(ax * ax + az * az), lb = sqrt(bx * bx + bz * bz);
        Real ab = ax * bx + az * bz;
        Real cr = ax * bz - az * bx;
        // theta1 = arccos(a.b / |a||b|), evaluated as atan2(|a x b|, a.b)
        Real th = atan2(fabs(cr), ab);
        Real sn = fabs(cr) / (la * lb);
        Real ratio = th < Real(1e-4) ? Real(1) + th * th / Real(6) : th / sn;
        Real dsp = la + lb;
        Real k1 = Real(0.25) * kb * (Real(-8) * ratio / dsp);
        Real dth = Real(2) * th;
        Real k2 = Real(0.25) * kb * (dth / dsp) * (dth / dsp);
        Real iab = Real(1) / (la * lb);
        Real dya_x = bx * iab - ab * ax * iab / (la * la), dya_z = bz * iab - ab * az * iab / (la * la);
        Real dyb_x = ax * iab - ab * bx * iab / (lb * lb), dyb_z = az * iab - ab * bz * iab / (lb * lb);
        Real gx = 0, gz = 0;
        if (k == mp) { gx += k1 * dya_x - k2 * ax / la; gz += k1 * dya_z - k2 * az / la; }
        if (k == m) {
          gx += k1 * (dyb_x - dya_x) - k2 * (bx / lb - ax / la);
          gz += k1 * (dyb_z - dya_z) - k2 * (bz / lb - az / la);
        }
        if (k == mq) { gx += -k1 * dyb_x + k2 * bx / lb; gz += -k1 * dyb_z + k2 * bz / lb; }
        F[0] -= gx;
        F[2] -= gz;
      }
    }
  } else {
    const int i0 = a.inc_off[k], ninc = a.inc_off[k + 1] - i0;
    if (lane < 16 && lane < ninc) {
      D3<Real> e = skalak_dual(a, a.inc[i0 + lane], k);
      F[0] -= e.d0; F[1] -= e.d1; F[2] -= e.d2;
    }
    // Helfrich vertex slots: 0 the marker, 1.. its distinct 1-ring
    // neighbours in the order of the incident faces and their vertices
    const int r0 = a.ring_off[k], nV = min(a.ring_off[k + 1] - r0 + 1, 16);
    int vs = 0, fs = 0, ds = 0;
    if (lane < nV) {
      vs = lane == 0 ? k : a.ring[r0 + lane - 1];
      fs = a.inc_off[vs];
      ds = a.inc_off[vs + 1] - fs;
    }
    int incl = ds;
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, sh);
      if (lane >= sh) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    Real* stg = hstage[threadIdx.x >> 5];
    DV<Real> K = {dc<Real>(0), dc<Real>(0), dc<Real>(0)};
    D3<Real> A = dc<Real>(0);
    for (int p0 = 0; p0 < total; p0 += 32) {
      const int p = p0 + lane;
      int S = 0;  // slot of pair p: the first whose inclusive prefix exceeds p
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, S + step - 1);
        if (v <= p) S += step;
      }
      const int vS = __shfl_sync(0xffffffffu, vs, S), fS = __shfl_sync(0xffffffffu, fs, S);
      const int eS = __shfl_sync(0xffffffffu, incl, S) - __shfl_sync(0xffffffffu, ds, S);
      if (p < total) {
        DV<Real> Kc;
        D3<Real> Ac;
        helfrich_term(a, vS, a.inc[fS + p - eS], k, Kc, Ac);
        const Real c[16] = {Kc.x.v, Kc.x.d0, Kc.x.d1, Kc.x.d2, Kc.y.v, Kc.y.d0, Kc.y.d1, Kc.y.d2,
                            Kc.z.v, Kc.z.d0, Kc.z.d1, Kc.z.d2, Ac.v,   Ac.d0,   Ac.d1,   Ac.d2};
#pragma unroll
        for (int q = 0; q < 16; ++q) stg[lane * 16 + q] = c[q];
      }
      __syncwarp();
      if (lane < nV) {  // this slot's pairs of the chunk, in face order
        const int lo = max(incl - ds, p0), hi = min(incl, p0 + 32);
        for (int q = lo; q < hi; ++q) {
          const Real* c = stg + (q - p0) * 16;
          K.x = K.x + D3<Real>{c[0], c[1], c[2], c[3]};
          K.y = K.y + D3<Real>{c[4], c[5], c[6], c[7]};
          K.z = K.z + D3<Real>{c[8], c[9], c[10], c[11]};
          A = A + D3<Real>{c[12], c[13], c[14], c[15]};
        }
      }
      __syncwarp();
    }
    if (lane < nV) {
      const Real kb = a.capr[a.ncaps + a.ncap[vs]];
      D3<Real> h = (kb * Real(0.125)) * (ddot(K, K) / A);
      F[0] -= h.d0; F[1] -= h.d1; F[2] -= h.d2;
    }
  }
  for (int d = 0; d < 3; ++d)
    for (int o = 16; o > 0; o >>= 1) F[d] += __shfl_xor_sync(0xffffffffu, F[d], o);
  if (lane == 0) {
    if (a.dim == 2) F[1] = 0;
    for (int d = 0; d < 3; ++d) a.F[3 * k + d] = F[d];
  }
}
template <class Real>
__global__ void k_node_forces(const __grid_constant__ IBArgs<Real> a) {
  if (blockIdx.x == 0 && threadIdx.x < 2) a.ctr[threadIdx.x] = 0;  // the brick compaction's counters
  node_forces_body(a, hw_blk());
}

// Coupling force on marker k from its fixed-point sum (integer totals, so
// the result does not depend on the order of the contributions).
template <class Real>
__device__ __forceinline__ void coupling_of(const IBArgs<Real>& a, int k, Real* out) {
  long long cpl[3];
  for (int d = 0; d < 3; ++d) cpl[d] = (long long)a.ncpl[3 * k + d];
  for (int d = 0; d < 3; ++d) {
    if constexpr (std::is_same<Real, float>::value)  // one rounding either way
      out[d] = __ll2float_rn(cpl[d]) * 0x1p-50f;
    else
      out[d] = (Real)((double)cpl[d] / CPL_SCALE);
  }
  if (a.dim == 2) out[1] = 0;
}

// ------------------------------------------------------------ spreading
template <class Real>
__device__ __forceinline__ Real peskin(Real r) {
  Real x = fabs(r);
  if (x <= Real(1)) return (Real(3) - Real(2) * x + sqrt(fmax(Real(0), Real(1) + Real(4) * x - Real(4) * x * x))) * Real(0.125);
  if (x <= Real(2)) return (Real(5) - Real(2) * x - sqrt(fmax(Real(0), Real(-7) + Real(12) * x - Real(4) * x * x))) * Real(0.125);
  return Real(0);
}

// Distinct bricks touched along one axis by the 4 support cells starting at base.
__device__ __forceinline__ int axis_bricks(int base, int n, int* out) {
  int m = 0;
  for (int s = 0; s < 4; ++s) {
    int c = ((base + s) % n + n) % n;
    int b = c / BRICK;
    bool dup = false;
    for (int j = 0; j < m; ++j) dup |= out[j] == b;
    if (!dup) out[m++] = b;
  }
  return m;
}

template <class Real>
__device__ __forceinline__ int node_bricks(const IBArgs<Real>& a, int l, int* out) {
  int bx[4], by[4], bz[4];
  int nxb = axis_bricks(a.xo[3 * l] - 1, a.G.nx, bx);
  int nyb = 1;
  by[0] = 0;
  if (a.dim == 3) nyb = axis_bricks(a.xo[3 * l + 1] - 1, a.G.ny, by);
  int nzb = axis_bricks(a.xo[3 * l + 2] - 1, a.G.nz, bz);
  int m = 0;
  for (int i = 0; i < nxb; ++i)
    for (int j = 0; j < nyb; ++j)
      for (int k = 0; k < nzb; ++k) out[m++] = (bz[k] * a.nby + by[j]) * a.nbx + bx[i];
  return m;
}

template <class Real>
__device__ __forceinline__ void brick_count_body(const IBArgs<Real>& a, const Blk& blk) {
  int l = blk.x * blockDim.x + threadIdx.x;
  if (l >= a.nn) return;
  int b[64];
  int m = node_bricks(a, l, b);
  for (int j = 0; j < m; ++j) atomicAdd(a.bcnt + b[j], 1);
}
template <class Real>
__global__ void k_brick_count(const __grid_constant__ IBArgs<Real> a) {
  brick_count_body(a, hw_blk());
}

// Bricks holding markers now or in the previous step join the active list;
// each claims a contiguous slot range for its marker list.
template <class Real>
__device__ __forceinline__ void brick_compact_body(const IBArgs<Real>& a, const Blk& blk) {
  int b = blk.x * blockDim.x + threadIdx.x;
  if (b >= a.nbricks) return;
  int c = a.bcnt[b];
  a.bflag[b] = c > 0;
  if (c == 0 && a.bprev[b] == 0) return;
  int i = atomicAdd(a.ctr, 1);
  a.bact[i] = b;
  a.boff[b] = atomicAdd(a.ctr + 1, c);
}
template <class Real>
__global__ void k_brick_compact(const __grid_constant__ IBArgs<Real> a) {
  brick_compact_body(a, hw_blk());
}

template <class Real>
__device__ __forceinline__ void brick_fill_body(const IBArgs<Real>& a, const Blk& blk) {
  int l = blk.x * blockDim.x + threadIdx.x;
  if (l >= a.nn) return;
  int b[64];
  int m = node_bricks(a, l, b);
  for (int j = 0; j < m; ++j) {
    int s = atomicAdd(a.bcur + b[j], 1);
    if (s >= a.bcnt[b[j]]) {  // count and fill disagree: flag, never write past the range
      atomicOr(a.status, (unsigned)ST_OVERFLOW);
      continue;
    }
    a.blist[a.boff[b[j]] + s] = l;
  }
}
template <class Real>
__global__ void k_brick_fill(const __grid_constant__ IBArgs<Real> a) {
  brick_fill_body(a, hw_blk());
}

// Each cell of an active brick sums F_l delta_h(x - X_l) over the brick's
// markers in ascending marker order (the list is sorted first, so the result
// does not depend on the order of the atomic slot claims).  Bricks that held
// markers in the previous step are visited too, so their cells return to zero.
template <class Real>
__device__ __forceinline__ void spread_body(const IBArgs<Real>& a, const Blk& blk) {
  constexpr int CH = 128;  // markers staged at a time
  __shared__ int list[512], sorted[512];
  __shared__ Real sW[CH][12];  // per marker: delta_h at the brick's 4 cells along x, y, z
  __shared__ Real sF[CH][3];
  const int nact = min(a.ctr[0], a.nbricks);
  const int BY = a.dim == 3 ? BRICK : 1;
  for (int ib = blk.x; ib < nact; ib += blk.gx) {
    const int b = a.bact[ib];
    if (b < 0 || b >= a.nbricks) continue;
    const int cnt = a.bcnt[b];
    const int off = a.boff[b];
    const int m = min(cnt, 512);
    if (cnt > 512 && threadIdx.x == 0) atomicOr(a.status, (unsigned)ST_OVERFLOW);
    for (int j = threadIdx.x; j < m; j += blockDim.x) list[j] = a.blist[off + j];
    __syncthreads();
    // rank sort (marker indices are distinct), so the sum runs in marker order
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      int v = list[j], r = 0;
      for (int i = 0; i < m; ++i) r += list[i] < v;
      sorted[r] = v;
    }
    __syncthreads();
    const int bx = b % a.nbx, by = (b / a.nbx) % a.nby, bz = b / (a.nbx * a.nby);
    const int ox = bx * BRICK, oy = by * BRICK, oz = bz * BRICK;
    const int lx = threadIdx.x % BRICK, ly = (threadIdx.x / BRICK) % BY, lz = threadIdx.x / (BRICK * BY);
    const int cx = ox + lx, cy = oy + ly, cz = oz + lz;
    const bool ok = threadIdx.x < BRICK * BY * BRICK && cx < a.G.nx && cy < a.G.ny && cz < a.G.nz;
    Real f[3] = {0, 0, 0};
    for (int j0 = 0; j0 < m; j0 += CH) {
      const int mc = min(CH, m - j0);
      // marker positions relative to the brick corner (nearest periodic
      // image) and the kernel weights of the brick's cells along each axis
      for (int j = threadIdx.x; j < mc; j += blockDim.x) {
        int l = sorted[j0 + j];
        Real r3[3];
        if constexpr (std::is_same<Real, float>::value) {
          // integer part wrapped to [-n/2, n/2) (the image nearest the brick)
          auto img = [](int k, int n) { return wrap_coord(k + n / 2, n) - n / 2; };
          r3[0] = (float)img(a.xo[3 * l] - ox, a.G.nx) + a.xr[3 * l];
          r3[1] = a.dim == 3 ? (float)img(a.xo[3 * l + 1] - oy, a.G.ny) + a.xr[3 * l + 1] : 0.0f;
          r3[2] = (float)(a.G.wall ? a.xo[3 * l + 2] - oz : img(a.xo[3 * l + 2] - oz, a.G.nz)) + a.xr[3 * l + 2];
        } else {
          double rx = a.X[3 * l] - ox, ry = a.X[3 * l + 1] - oy, rz = a.X[3 * l + 2] - oz;
          rx -= a.G.nx * floor(rx / a.G.nx + 0.5);
          if (a.dim == 3) ry -= a.G.ny * floor(ry / a.G.ny + 0.5); else ry = 0;
          if (!a.G.wall) rz -= a.G.nz * floor(rz / a.G.nz + 0.5);
          r3[0] = (Real)rx;
          r3[1] = (Real)ry;
          r3[2] = (Real)rz;
        }
        // delta_h vanishes outside |r| < 2 (peskin returns 0 there)
  #pragma unroll
        for (int d = 0; d < 3; ++d)
  #pragma unroll
          for (int o = 0; o < BRICK; ++o) sW[j][4 * d + o] = peskin((Real)o - r3[d]);
        Real cp[3];
        coupling_of(a, l, cp);  // F_mem = F_s + F_b + F_c (eq. MembraneForces)
        for (int d = 0; d < 3; ++d) sF[j][d] = a.F[3 * l + d] + cp[d];
      }
      __syncthreads();
      if (ok) {  // summed in marker order across the chunks
        for (int j = 0; j < mc; ++j) {
          Real wgt = sW[j][lx] * sW[j][8 + lz];
          if (a.dim == 3) wgt *= sW[j][4 + ly];
          if (wgt == Real(0)) continue;  // outside the support
          for (int d = 0; d < 3; ++d) f[d] += wgt * sF[j][d];
        }
      }
      __syncthreads();
    }
    if (ok) {
      long long c = ((long long)cz * a.G.ny + cy) * a.G.nx + cx;
      for (int d = 0; d < 3; ++d) a.fib[d * a.G.P + c] = f[d];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a.bprev[b] = cnt;
      a.bcnt[b] = 0;
      a.bcur[b] = 0;
    }
    __syncthreads();
  }
}
template <class Real>
__global__ void k_spread(const __grid_constant__ IBArgs<Real> a) {
  spread_body(a, hw_blk());
}

// ------------------------------------------------------------ interpolation
// One warp per marker: v(t+1) = (j' + F/2)/rho' on the 4^d support cells
// from the streamed populations and the force of the step, weighted by
// delta_h, reduced over the warp; then X += U (explicit Euler).
template <class L, int MODE>
__device__ __forceinline__ void interp_advect_body(const IBArgs<typename Prec<MODE>::Real>& a,
                                                   const typename Prec<MODE>::Store* lo, const Blk& blk) {
  using Real = typename Prec<MODE>::Real;
  int l = (blk.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (l >= a.nn) return;
  const Geo G = a.G;
  const int bb[3] = {a.xo[3 * l] - 1, a.xo[3 * l + 1] - 1, a.xo[3 * l + 2] - 1};
  // delta_h along each axis at the 4 support offsets: lane 4 d + o
  Real wax = 0;
  if (lane < 12) {
    const int d = lane >> 2, o = lane & 3;
    if (d != 1 || a.dim == 3) wax = peskin(-node_off(a, l, d, bb[d] + o));
  }
  const int ncell = a.dim == 3 ? 64 : 16;
  // the lane's two support cells: weights and addresses first, so that all
  // their loads are in flight together (a cell of weight 0 reads cell 0)
  Real w[2];
  int cx[2], cy[2], cz[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int s = lane + 32 * h;
    const int ox = s % 4, oy = a.dim == 3 ? (s / 4) % 4 : 0, oz = a.dim == 3 ? s / 16 : (s / 4) % 4;
    w[h] = __shfl_sync(0xffffffffu, wax, ox) * __shfl_sync(0xffffffffu, wax, 8 + oz);
    if (a.dim == 3) w[h] *= __shfl_sync(0xffffffffu, wax, 4 + oy);
    const int px = bb[0] + ox, py = a.dim == 3 ? bb[1] + oy : 0, pz = bb[2] + oz;
    const bool ok = s < ncell && w[h] != Real(0) && !(G.wall && (pz < 0 || pz >= G.nz));
    if (!ok) w[h] = 0;
    cx[h] = ok ? wrap_coord(px, G.nx) : 0;
    cy[h] = ok ? wrap_coord(py, G.ny) : 0;
    cz[h] = ok ? wrap_coord(pz, G.nz) : 0;
  }
  Real U[3] = {0, 0, 0};
  if (a.M) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const Nbr<L> nb(G, cx[h], cy[h], cz[h]);
      const long long self = nb.self;
      Real r = 0, j[3] = {0, 0, 0};
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        EqCell<L, Real> e;
        e.load_f(a.M, G.P32, nb.src(i));
        const Real fi = e.f(nb.bounce(i) ? L::opp(i) : i);
        r += fi;
        if (L::cx(i)) j[0] += L::cx(i) > 0 ? fi : -fi;
        if (L::cy(i)) j[1] += L::cy(i) > 0 ? fi : -fi;
        if (L::cz(i)) j[2] += L::cz(i) > 0 ? fi : -fi;
      }
      Real ft[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) ft[d] = a.ftot[d * G.P + self];
      Real rho = Real(1) + r;
      if (w[h] != Real(0))
        for (int d = 0; d < 3; ++d) U[d] += w[h] * (j[d] + Real(0.5) * ft[d]) / rho;
    }
  } else {
    // the populations of both support cells (and their forces) are all
    // requested before the first sum, so their latencies overlap
    Real fv[2][L::Q], ft[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const Nbr<L> nb(G, cx[h], cy[h], cz[h]);
#pragma unroll
      for (int i = 0; i < L::Q; ++i) fv[h][i] = to_real(__ldg(lo + nb.off(i, plane_f<L>(i), plane_f<L>(L::opp(i)), G.P32)));
#pragma unroll
      for (int d = 0; d < 3; ++d) ft[h][d] = __ldg(a.ftot + d * G.P + nb.self);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      Real r = 0, j[3] = {0, 0, 0};
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const Real fi = fv[h][i];
        r += fi;
        if (L::cx(i)) j[0] += L::cx(i) > 0 ? fi : -fi;
        if (L::cy(i)) j[1] += L::cy(i) > 0 ? fi : -fi;
        if (L::cz(i)) j[2] += L::cz(i) > 0 ? fi : -fi;
      }
      Real rho = Real(1) + r;
      if (w[h] != Real(0))
        for (int d = 0; d < 3; ++d) U[d] += w[h] * (j[d] + Real(0.5) * ft[h][d]) / rho;
    }
  }
  for (int d = 0; d < 3; ++d)
    for (int o = 16; o > 0; o >>= 1) U[d] += __shfl_xor_sync(0xffffffffu, U[d], o);
  // lane 0's totals (each lane's butterfly sums in its own order)
  for (int d = 0; d < 3; ++d) U[d] = __shfl_sync(0xffffffffu, U[d], 0);
  if (a.dim == 2) U[1] = 0;
  if (lane == 0 && !(fabs(U[0]) < Real(0.5) && fabs(U[1]) < Real(0.5) && fabs(U[2]) < Real(0.5)))
    atomicOr(a.status, (unsigned)ST_MARKER_JUMP);
  if (lane < 3) {  // lane d advances coordinate d
    const int d = lane;
    const Real Ud = d == 0 ? U[0] : (d == 1 ? U[1] : U[2]);
    const double Xn = a.X[3 * l + d] + (double)Ud;
    a.X[3 * l + d] = Xn;
    double v = fmax(-1e8, fmin(1e8, Xn));
    atomicMin(a.box + d, (int)floor(v));
    atomicMin(a.box + 3 + d, -(int)ceil(v));
    split_coord(Xn, a.xo + 3 * l + d, a.xr + 3 * l + d);
  }
}
template <class L, int MODE>
__global__ void k_interp_advect(const __grid_constant__ IBArgs<typename Prec<MODE>::Real> a,
                                const typename Prec<MODE>::Store* lo) {
  interp_advect_body<L, MODE>(a, lo, hw_blk());
}

// FP64 capsule measures: 2D enclosed area (shoelace in the internal x-z
// plane); 3D surface area and enclosed volume (divergence theorem).
__global__ void k_capsule_measures(const double* X, const int* E, const int* ecap, int ne, int NV, int ncap,
                                   double* out /* [ncap][2] */);
