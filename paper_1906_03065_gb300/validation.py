"""The paper's 2D validation experiments on the GPU (Sec. 4), run as batches
of independent lattices through the library.

* Sec. 4.1: an initially circular capsule (R = 20) at the centre of a 12R x
  6R periodic domain on a C1/C2 interface; alpha = 2, kappa_c = 1e-2;
  kappa_s in {1e-3, 1e-2, 1e-1}, kappa_b in {1e-4, 1e-2}; the symmetric case
  kappa_1 = kappa_2 = 8e-3 with kappa_3 from 5e-4 to 1e-2, the asymmetric
  case kappa_1 = 8e-3, kappa_2 = 2e-3 with kappa_3 from 5e-4 to 8e-3 (steps
  of 5e-4); the result is the Taylor deformation D = (L - B)/(L + B) of the
  relaxed capsule, and of the pure liquid lens (no membrane) beside it.
* Sec. 4.1, Galilean invariance: every fluid starts with a uniform U_x0 in
  {1e-4, 1e-3, 1e-2}; the relaxed shapes, with the drift removed, are the
  stationary one.
* Sec. 4.2: a capillary bridge of C2 (R x 31R/10) between two capsules at
  (9R/2, 3R) and (15R/2, 3R) in C1; kappa_1 in {1e-3, 3e-3, 9e-3}, kappa_2 =
  3e-3, kappa_3 = 6e-3, kappa_b = 1e-2; the result is the capsules' aspect
  ratio L_c / H_c against kappa_s.

Readings (the paper prints no recipe for these measures): L and B are the
axes of the ellipse with the same second moments of area as the region the
markers enclose; L_c and H_c are the capsule's extents along and across the
line joining the capsules.  The periodic domain carries two flat C1/C2
interfaces (C1 in the upper half), each of tanh profile.  Only host-side
set-up and measurement live here; every step runs in the library's kernels.
The paper's reference shapes (Surface Evolver) exist only in its figures and
are not reproduced.
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as W

R_PAPER = 20.0


def _ring_nodes(R: float) -> int:
    """Markers one lattice unit apart on the initial circle (Sec. 3.2)."""
    return int(round(2 * math.pi * R))


def capsule_at_interface(kappa, ks: float, kb: float, U: float = 0.0, R: float = R_PAPER,
                         membrane: bool = True, storage: str = "f64") -> W.Workload:
    """Sec. 4.1 set-up: 12R x 6R periodic D2Q9 lattice, capsule of radius R
    at the centre on the interface, alpha = 2, kappa_c = 1e-2, tau = Gamma =
    1 (Sec. 3.1), uniform initial velocity U along x."""
    nx, ny = int(12 * R), int(6 * R)
    p = W.Params(dim=2, nx=nx, ny=ny, nz=1, storage=storage, alpha=2.0, kappa1=kappa[0], kappa2=kappa[1],
                 kappa3=kappa[2], kappa_c=1e-2, dc=16.0, interface_pos=ny / 2.0, u0=(U, 0.0, 0.0))
    mems = []
    if membrane:
        m = W.ring(_ring_nodes(R), R, (nx / 2.0, ny / 2.0))
        m.ks, m.kb = ks, kb
        mems.append(m)
    return W.Workload(f"paper_capsule_k{kappa[0]:g}_{kappa[1]:g}_{kappa[2]:g}_ks{ks:g}_kb{kb:g}_U{U:g}", p, mems)


def _band(y, lo: float, hi: float, alpha: float):
    """Indicator of lo <= y < hi on a periodic axis of length ny, with tanh
    profiles (eq. CmProfile) across both edges."""
    return 0.5 * (np.tanh((y - lo) / (2 * alpha)) - np.tanh((y - hi) / (2 * alpha)))


def initial_fields(wl: W.Workload, bridge=None):
    """C1, C2, C3 (3, ncells) of a Sec. 4 set-up: C3 inside the capsules
    (tanh of the distance to each circle), then C1 above and C2 below the
    mid-height (two periodic interfaces), or, with ``bridge`` = (x0, x1, y0,
    y1), C2 in that rectangle and C1 around it."""
    p = wl.params
    y, x = np.meshgrid(np.arange(p.ny, dtype=float), np.arange(p.nx, dtype=float), indexing="ij")
    a = p.alpha
    C3 = np.zeros_like(x)
    for m in wl.membranes:
        c = m.X.mean(axis=0)
        R = float(np.linalg.norm(m.X[:, :2] - c[:2], axis=1).mean())
        C3 = np.maximum(C3, 0.5 * (1 + np.tanh((R - np.hypot(x - c[0], y - c[1])) / (2 * a))))
    if bridge is None:
        # C1 in [ny/2, ny): interfaces at ny/2 and at 0 = ny
        s = _band(y, p.ny / 2.0, p.ny, a) + _band(y, p.ny / 2.0 - p.ny, 0.0, a)
        C1, C2 = (1 - C3) * s, (1 - C3) * (1 - s)
    else:
        x0, x1, y0, y1 = bridge
        r = _band(x, x0, x1, a) * _band(y, y0, y1, a)
        C2, C1 = (1 - C3) * r, (1 - C3) * (1 - r)
    return np.stack([C1.ravel(), C2.ravel(), C3.ravel()])


def capillary_bridge(kappa1: float, ks: float, kb: float = 1e-2, R: float = R_PAPER, storage: str = "f64"):
    """Sec. 4.2 set-up: two capsules of radius R at (9R/2, 3R) and (15R/2, 3R)
    in C1, a C2 bridge of 2S x H_b = R x 31R/10 at the centre; kappa_2 =
    3e-3, kappa_3 = 6e-3, alpha = 2, kappa_c = 1e-2.  Returns the workload
    and the bridge rectangle."""
    nx, ny = int(12 * R), int(6 * R)
    p = W.Params(dim=2, nx=nx, ny=ny, nz=1, storage=storage, alpha=2.0, kappa1=kappa1, kappa2=3e-3,
                 kappa3=6e-3, kappa_c=1e-2, dc=16.0, interface_pos=-1.0)
    mems = []
    for xc in (4.5 * R, 7.5 * R):
        m = W.ring(_ring_nodes(R), R, (xc, 3 * R))
        m.ks, m.kb = ks, kb
        mems.append(m)
    wl = W.Workload(f"paper_bridge_k1{kappa1:g}_ks{ks:g}", p, mems)
    return wl, (nx / 2.0 - R / 2, nx / 2.0 + R / 2, 3 * R - 31 * R / 20, 3 * R + 31 * R / 20)


def area_moments(X: np.ndarray):
    """Area, centroid and central second-moment tensor [[Ixx, Ixy], [Ixy,
    Iyy]] (Ixx = integral of (x - cx)^2) of the polygon X (n, 2+), counter-
    clockwise, by the polygon (Green's theorem) formulas."""
    x, y = X[:, 0], X[:, 1]
    x1, y1 = np.roll(x, -1), np.roll(y, -1)
    cr = x * y1 - x1 * y
    A = 0.5 * cr.sum()
    cx = ((x + x1) * cr).sum() / (6 * A)
    cy = ((y + y1) * cr).sum() / (6 * A)
    ixx = ((x * x + x * x1 + x1 * x1) * cr).sum() / 12 - A * cx * cx
    iyy = ((y * y + y * y1 + y1 * y1) * cr).sum() / 12 - A * cy * cy
    ixy = ((x * y1 + 2 * x * y + 2 * x1 * y1 + x1 * y) * cr).sum() / 24 - A * cx * cy
    return A, (cx, cy), np.array([[ixx, ixy], [ixy, iyy]])


def taylor_deformation(X: np.ndarray) -> float:
    """D = (L - B)/(L + B) of the ellipse with the polygon's second moments
    of area: its axis ratio L/B is the square root of the tensor's
    eigenvalue ratio."""
    _, _, M = area_moments(X)
    ev = np.linalg.eigvalsh(M)
    r = math.sqrt(ev[1] / ev[0])
    return (r - 1) / (r + 1)


def lens_deformation(psi: np.ndarray, shape) -> float:
    """D of a pure liquid lens from the second moments of its C3 field."""
    ps = psi.reshape(shape)
    y, x = np.meshgrid(np.arange(shape[0], dtype=float), np.arange(shape[1], dtype=float), indexing="ij")
    w = ps / ps.sum()
    cx, cy = (w * x).sum(), (w * y).sum()
    M = np.array([[(w * (x - cx) ** 2).sum(), (w * (x - cx) * (y - cy)).sum()],
                  [(w * (x - cx) * (y - cy)).sum(), (w * (y - cy) ** 2).sum()]])
    ev = np.linalg.eigvalsh(M)
    r = math.sqrt(ev[1] / ev[0])
    return (r - 1) / (r + 1)


def aspect_ratio(X: np.ndarray) -> float:
    """L_c / H_c: the capsule's extent along x (the line joining the bridge's
    capsules) over its extent along y."""
    return float((X[:, 0].max() - X[:, 0].min()) / (X[:, 1].max() - X[:, 1].min()))


def tensions(kappa, alpha: float = 2.0):
    """gamma_12, gamma_13, gamma_23 of eq. SurfaceTension."""
    k1, k2, k3 = kappa
    return alpha * (k1 + k2) / 6, alpha * (k1 + k3) / 6, alpha * (k2 + k3) / 6


def relax(wls, steps: int, fields=None, check_every: int = 1000, tol: float = 0.0, device="cuda:0"):
    """Relax the workloads (one lattice size) together as one batch from the
    given initial fields (default initial_fields); returns the batch."""
    from . import Batch
    b = Batch(wls, device=device)
    for i, wl in enumerate(wls):
        b[i].init(initial_fields(wl) if fields is None else fields[i], None)
    b.run(steps, check_every, tol)
    return b


def symmetric_case():
    """Sec. 4.1 symmetric case: kappa_1 = kappa_2 = 8e-3, kappa_3 = 5e-4 .. 1e-2."""
    return [(8e-3, 8e-3, 5e-4 * k) for k in range(1, 21)]


def asymmetric_case():
    """Sec. 4.1 asymmetric case: kappa_1 = 8e-3, kappa_2 = 2e-3, kappa_3 = 5e-4 .. 8e-3."""
    return [(8e-3, 2e-3, 5e-4 * k) for k in range(1, 17)]


def deformation_sweep(cases, ks_list=(1e-3, 1e-2, 1e-1), kb_list=(1e-4, 1e-2), steps: int = 40000,
                      lens: bool = True, device="cuda:0", storage: str = "f32"):
    """Taylor deformation of the relaxed capsule for every (kappa, ks, kb),
    relaxed together as one batch, and of the pure lens for every kappa, as
    a second batch.  Returns rows of (kappa, ratio g12/g13, g13/g23, ks, kb,
    D), the capsules in (ks, kb, kappa) order, then the lenses."""
    rows = []
    combos = [(ks, kb, k) for ks in ks_list for kb in kb_list for k in cases]
    if combos:
        wls = [capsule_at_interface(k, ks, kb, storage=storage) for ks, kb, k in combos]
        b = relax(wls, steps, device=device)
        for i, (ks, kb, k) in enumerate(combos):
            g12, g13, g23 = tensions(k)
            rows.append({"kappa": k, "g12/g13": g12 / g13, "g13/g23": g13 / g23, "ks": ks, "kb": kb,
                         "D": taylor_deformation(b[i].nodes(0))})
        del b
    if lens:
        wls = [capsule_at_interface(k, 0.0, 0.0, membrane=False, storage=storage) for k in cases]
        fields = []
        for k in cases:
            m = W.ring(_ring_nodes(R_PAPER), R_PAPER, (120.0, 60.0))
            tmp = W.Workload("lens", wls[0].params, [m])
            fields.append(initial_fields(tmp))
        b = relax(wls, steps, fields=fields, device=device)
        for i, k in enumerate(cases):
            g12, g13, g23 = tensions(k)
            rows.append({"kappa": k, "g12/g13": g12 / g13, "g13/g23": g13 / g23, "ks": None, "kb": None,
                         "D": lens_deformation(b[i].field("psi"), (wls[i].params.ny, wls[i].params.nx))})
        del b
    return rows


def galilean_runs(kappa=(8e-3, 8e-3, 5e-4), ks: float = 1e-3, kb: float = 1e-2, U_list=(1e-4, 1e-3, 1e-2),
                  steps: int = 20000, R: float = R_PAPER, device="cuda:0", storage: str = "f32"):
    """Sec. 4.1, Galilean invariance: the capsule with every fluid started
    at a uniform U_x0, relaxed beside the stationary run (U = 0) as one
    batch.  Returns rows of (U, the mean marker displacement from the
    stationary run, U * steps, the largest distance between corresponding
    markers of the two shapes with each centroid removed, D of both)."""
    wls = [capsule_at_interface(kappa, ks, kb, U=U, R=R, storage=storage) for U in (0.0,) + tuple(U_list)]
    b = relax(wls, steps, device=device)
    X0 = b[0].nodes(0)

    def centred(X):
        return X[:, :2] - X[:, :2].mean(axis=0)

    rows = []
    for i, U in enumerate(U_list, start=1):
        X = b[i].nodes(0)
        rows.append({"U": U, "drift": (X[:, :2] - X0[:, :2]).mean(axis=0).tolist(), "U_steps": U * steps,
                     "shape_dev": float(np.abs(centred(X) - centred(X0)).max()),
                     "D": taylor_deformation(X), "D_stationary": taylor_deformation(X0)})
    del b
    return rows


def bridge_sweep(kappa1_list=(1e-3, 3e-3, 9e-3), ks_list=(1e-3, 1e-2, 1e-1), steps: int = 20000,
                 device="cuda:0", storage: str = "f32"):
    """Sec. 4.2: aspect ratio L_c / H_c of both capsules of the capillary
    bridge for every (kappa_1, ks), relaxed as one batch.  Returns rows of
    (kappa_1, ks, [L_c / H_c of capsule 0, of capsule 1])."""
    from . import Batch
    cases = [(k1, ks) for k1 in kappa1_list for ks in ks_list]
    built = [capillary_bridge(k1, ks, storage=storage) for k1, ks in cases]
    b = Batch([wl for wl, _ in built], device=device)
    for i, (wl, rect) in enumerate(built):
        b[i].init(initial_fields(wl, bridge=rect), None)
    b.run(steps, 1000, 0.0)
    rows = []
    for i, (k1, ks) in enumerate(cases):
        rows.append({"kappa1": k1, "ks": ks, "aspect": [aspect_ratio(b[i].nodes(m)) for m in range(2)]})
    del b
    return rows
