"""Seeded synthetic inputs: lattice parameters and membrane geometry.

This module holds no arithmetic of the method itself (no equilibria, no
chemical potentials, no forces).  It only produces the *inputs* of a run:
lattice sizes and physical parameters, membrane meshes (a closed ring of
Lagrangian markers in 2D, a subdivided icosahedron in 3D) and seeded random
perturbations.  Both the CUDA path and the CPU oracle consume these inputs.

Workload recipes (lattice units, dx = dt = 1, Sec. 3.1 of the paper):

* ``capsule_2d``  -- D2Q9, 64x64 periodic, one circular capsule of radius 12
  (76 markers) centred on a flat C1/C2 interface; the paper's own set-up is a
  capsule at a fluid-fluid interface (Sec. 4.1), here at a smaller size.
* ``capsule_3d``  -- D3Q19, 128^3, walls at the two ends of z, periodic in x
  and y; flat C1/C2 interface at z = 64 and a spherical capsule of radius 20
  (icosphere level 4: 2562 nodes, 5120 triangles) centred on it.
* ``bridge_3d``   -- D3Q19 192x128x128: two capsules 48 apart along x with a
  C1 cylinder between them in C2 (the 3D analogue of the paper's capillary
  bridge, Sec. 4.2).
* ``sweep_3d``    -- 64 independent cubic lattices of edge 48..96, each a
  capsule on an interface with seeded fluid and membrane parameters (the
  parameter sweeps behind the paper's Sec. 4 figures, run as one batch).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import List, Optional

import numpy as np

STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
MEM_RING2D = 0
MEM_TRI3D = 1


@dataclass
class Params:
    dim: int = 2
    nx: int = 64
    ny: int = 64
    nz: int = 1
    wall_last: int = 0          # 1: walls at both ends of the last axis
    storage: str = "f64"
    tau: float = 1.0
    tau_phi: float = 1.0
    tau_psi: float = 1.0
    gamma_phi: float = 1.0
    gamma_psi: float = 1.0
    alpha: float = 1.0
    kappa1: float = 0.01
    kappa2: float = 0.01
    kappa3: float = 0.01
    kappa_c: float = 0.01
    dc: float = 8.0             # clamp distance of the membrane profile
    u0: tuple = (0.0, 0.0, 0.0)
    interface_pos: float = 32.0  # flat C1/C2 interface along the last axis
    forcing: str = "edm"        # "edm": exact difference method (the paper); "guo": Guo forcing
    state: str = "populations"  # "populations", or "moments": 11 stored moments per cell (tau = 1)
    force_form: str = "potential"  # free-energy force: "potential" or "pressure_tensor" (App. A)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def as_dict(self):
        d = asdict(self)
        d["u0"] = list(self.u0)
        return d


@dataclass
class Membrane:
    kind: int
    X: np.ndarray                    # (n, 3) float64; z = 0 in 2D
    elems: Optional[np.ndarray]      # (ne, 2|3) int32
    ks: float = 0.0                  # 2D stretching modulus
    kb: float = 0.0                  # bending modulus (2D and 3D)
    G: float = 0.0                   # 3D Skalak shear modulus
    C: float = 1.0                   # 3D Skalak area-dilation ratio


@dataclass
class Workload:
    name: str
    params: Params
    membranes: List[Membrane] = field(default_factory=list)
    steps: int = 100


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------
def ring(n: int, radius: float, centre, phase: float = 0.0) -> Membrane:
    """Closed ring of ``n`` markers, counter-clockwise (outward normal = right
    of the tangent).  Segment l joins marker l to marker l+1 (mod n)."""
    k = np.arange(n, dtype=np.float64)
    th = phase + 2.0 * math.pi * k / n
    X = np.zeros((n, 3))
    X[:, 0] = centre[0] + radius * np.cos(th)
    X[:, 1] = centre[1] + radius * np.sin(th)
    elems = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1).astype(np.int32)
    return Membrane(MEM_RING2D, X, elems)


def icosphere(level: int, radius: float, centre) -> Membrane:
    """Icosahedron subdivided ``level`` times (each triangle split in four at
    edge midpoints) and projected on a sphere.  Triangles are counter-clockwise
    seen from outside.  level 3: 642 nodes / 1280 triangles, level 4: 2562 / 5120."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    faces = list(F)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    P = np.array(verts)
    T = np.array(faces, dtype=np.int32)
    # orient outward
    a, b, c = P[T[:, 0]], P[T[:, 1]], P[T[:, 2]]
    s = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c)
    flip = s < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    X = np.asarray(centre, dtype=np.float64)[None, :] + radius * P
    return Membrane(MEM_TRI3D, X, T)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def capsule_2d(storage: str = "f64") -> Workload:
    """64x64 periodic D2Q9; tau = 1 and Gamma = 0.2 so that M = Gamma(tau - 1/2)
    = 0.1 (Sec. 3.1, eq. RelaxationTimes); alpha = 1; kappa_1..3 = 0.01;
    kappa_c = 0.01; ring of 76 markers, R = 12 at (32, 32); ks = 0.05, kb = 0.001."""
    p = Params(dim=2, nx=64, ny=64, nz=1, storage=storage, gamma_phi=0.2,
               gamma_psi=0.2, alpha=1.0, kappa1=0.01, kappa2=0.01, kappa3=0.01,
               kappa_c=0.01, dc=8.0, interface_pos=32.0)
    m = ring(76, 12.0, (32.0, 32.0))
    m.ks, m.kb = 0.05, 0.001
    return Workload("capsule_2d_64x64_ring76", p, [m], steps=2000)


def capsule_3d(storage: str = "f32", n: int = 128, level: int = 4,
               radius: float = 20.0) -> Workload:
    """n^3 D3Q19, walls at both ends of z; kappa = (0.01, 0.02, 0.015), alpha = 2,
    kappa_c = 0.01, tau = Gamma = 1 (Sec. 3.1); icosphere capsule on the
    interface, Skalak G = 0.01, C = 1, Helfrich kb = 0.005."""
    c = n / 2.0
    p = Params(dim=3, nx=n, ny=n, nz=n, wall_last=1, storage=storage,
               alpha=2.0, kappa1=0.01, kappa2=0.02, kappa3=0.015,
               kappa_c=0.01, dc=16.0, interface_pos=c)
    m = icosphere(level, radius, (c, c, c))
    m.G, m.C, m.kb = 0.01, 1.0, 0.005
    return Workload(f"capsule_3d_{n}^3_ico{level}", p, [m], steps=20000)


def bridge_3d(storage: str = "f16", seed: int = 0) -> Workload:
    """192x128x128 D3Q19, walls in z; two capsules R = 20, 48 apart along x,
    Skalak G ~ U[0.005, 0.02] (seeded), kappa = 0.01 each, kb = 0.005."""
    rng = np.random.default_rng(seed)
    p = Params(dim=3, nx=192, ny=128, nz=128, wall_last=1, storage=storage,
               alpha=2.0, kappa1=0.01, kappa2=0.01, kappa3=0.01, kappa_c=0.01,
               dc=16.0, interface_pos=-1.0)
    mems = []
    for xc in (72.0, 120.0):
        m = icosphere(4, 20.0, (xc, 64.0, 64.0))
        m.G, m.C, m.kb = float(rng.uniform(0.005, 0.02)), 1.0, 0.005
        mems.append(m)
    return Workload("bridge_3d_192x128x128", p, mems, steps=30000)


def small_2d(storage: str = "f64", nx: int = 40, ny: int = 36, nodes: int = 50,
             radius: float = 8.0, centre=(20.3, 17.6), u0=(0.0, 0.0, 0.0)) -> Workload:
    """Ragged 2D case (sizes not multiples of a tile) used for parity."""
    p = Params(dim=2, nx=nx, ny=ny, nz=1, storage=storage, gamma_phi=0.2,
               gamma_psi=0.2, alpha=1.0, kappa1=0.012, kappa2=0.008, kappa3=0.01,
               kappa_c=0.01, dc=8.0, interface_pos=17.0, u0=tuple(u0))
    m = ring(nodes, radius, centre, phase=0.1)
    m.ks, m.kb = 0.05, 0.002
    return Workload(f"small_2d_{nx}x{ny}", p, [m], steps=300)


def small_3d(storage: str = "f32", nx: int = 40, ny: int = 36, nz: int = 34,
             level: int = 2, radius: float = 7.0, centre=(20.2, 18.1, 17.3),
             wall: int = 1) -> Workload:
    """Ragged 3D case with walls in z, icosphere level 2 (162 nodes)."""
    p = Params(dim=3, nx=nx, ny=ny, nz=nz, wall_last=wall, storage=storage,
               alpha=1.0, kappa1=0.01, kappa2=0.02, kappa3=0.015, kappa_c=0.01,
               dc=8.0, interface_pos=17.0)
    m = icosphere(level, radius, centre)
    m.G, m.C, m.kb = 0.01, 1.0, 0.005
    return Workload(f"small_3d_{nx}x{ny}x{nz}", p, [m], steps=200)


def sweep_3d(n_inst: int = 64, seed: int = 1, storage: str = "f16",
             edges=(48, 64, 80, 96)) -> List[Workload]:
    """Parameter sweep of independent cubic 3D lattices, drawn in order from
    numpy's PCG64 with ``seed``: edge ~ U{edges}; capsule radius R = edge *
    U[0.15, 0.25] on an icosphere of level 3 if R < 15 else 4; kappa_1,
    kappa_2, kappa_3 ~ U[0.005, 0.03] each; Skalak G ~ U[0.002, 0.05].  Every
    instance has the layout of ``capsule_3d`` (walls at the two ends of z, a
    flat C1/C2 interface at mid-height and the capsule centred on it) with
    C = 1, kb = 0.005, alpha = 2, kappa_c = 0.01, dc = 16, tau = 1 and
    Gamma_phi = Gamma_psi = 0.5 (mobility 0.25): with Gamma = 1 and alpha = 2
    the order-parameter update diverges for kappa_i above about 0.025."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        n = int(rng.choice(np.asarray(edges)))
        R = float(n * rng.uniform(0.15, 0.25))
        level = 3 if R < 15 else 4
        k1, k2, k3 = (float(v) for v in rng.uniform(0.005, 0.03, 3))
        G = float(rng.uniform(0.002, 0.05))
        c = n / 2.0
        p = Params(dim=3, nx=n, ny=n, nz=n, wall_last=1, storage=storage, alpha=2.0, gamma_phi=0.5,
                   gamma_psi=0.5, kappa1=k1, kappa2=k2, kappa3=k3, kappa_c=0.01, dc=16.0, interface_pos=c)
        m = icosphere(level, R, (c, c, c))
        m.G, m.C, m.kb = G, 1.0, 0.005
        out.append(Workload(f"sweep{i}_{n}^3_R{R:.1f}_ico{level}", p, [m], steps=20000))
    return out


def small_sweep_3d(n_inst: int = 4, seed: int = 7, storage: str = "f32") -> List[Workload]:
    """Small uneven 3D instances for parity of the batched path: x, y ~
    U{24..36}, z ~ U{22..30} (walls in z), capsule R = min(size) * U[0.15,
    0.22] on an icosphere of level 2 centred (off the grid) on the interface
    at mid-height, kappa_i ~ U[0.005, 0.03], G ~ U[0.002, 0.05], alpha = 1,
    dc = 8."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        nx, ny = (int(v) for v in rng.integers(24, 37, 2))
        nz = int(rng.integers(22, 31))
        R = float(min(nx, ny, nz) * rng.uniform(0.15, 0.22))
        k1, k2, k3 = (float(v) for v in rng.uniform(0.005, 0.03, 3))
        G = float(rng.uniform(0.002, 0.05))
        ctr = (nx / 2.0 + 0.3, ny / 2.0 - 0.2, nz / 2.0 + 0.1)
        p = Params(dim=3, nx=nx, ny=ny, nz=nz, wall_last=1, storage=storage, alpha=1.0,
                   kappa1=k1, kappa2=k2, kappa3=k3, kappa_c=0.01, dc=8.0, interface_pos=nz / 2.0)
        m = icosphere(2, R, ctr)
        m.G, m.C, m.kb = G, 1.0, 0.005
        out.append(Workload(f"small_sweep{i}_{nx}x{ny}x{nz}", p, [m], steps=200))
    return out


def jitter_nodes(m: Membrane, amp: float, seed: int) -> Membrane:
    """Seeded uniform jitter of the marker positions (in-plane only for rings)."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(-amp, amp, size=m.X.shape)
    if m.kind == MEM_RING2D:
        d[:, 2] = 0.0
    return Membrane(m.kind, m.X + d, None if m.elems is None else m.elems.copy(),
                    m.ks, m.kb, m.G, m.C)


def random_fields(p: Params, seed: int, amp: float = 0.02):
    """Seeded smooth-ish random concentration fields C1, C2, C3 (summing to a
    density near 1) and a small random velocity, shaped (3, ncells) each."""
    rng = np.random.default_rng(seed)
    n = p.ncells
    C3 = np.clip(rng.uniform(0.0, 1.0, n), 0, 1) * 0.2
    s = rng.uniform(0.0, 1.0, n)
    C1 = (1.0 - C3) * s
    C2 = (1.0 - C3) * (1.0 - s)
    C = np.stack([C1, C2, C3]) * (1.0 + rng.uniform(-amp, amp, n))[None, :]
    u = rng.uniform(-amp, amp, (3, n)) * 0.05
    if p.dim == 2:
        u[2] = 0.0
    return C, u
