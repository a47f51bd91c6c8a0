"""Pins of the oracle's lattice Boltzmann part (no GPU).

* chemical potentials are the variational derivatives of the discrete free
  energy (eqs. LandauFE, CouplingE, ChemPot; App. A) and vanish in the bulk
  minima (eq. Minimizers),
* the collision moves mass, momentum and the order-parameter moments exactly
  as the exact-difference and BGK schemes require (eqs. LBE, EDF,
  VelCorrection, ActualFluidVel), checked by un-streaming one step,
* per-component mass conservation, integer-shift equivariance, Galilean
  translation of a droplet (Sec. 4.1),
* a relaxed flat interface has the tanh profile and surface tension
  alpha (kappa_m + kappa_n)/6 (eqs. CmProfile, SurfaceTension); a droplet obeys
  the Laplace law.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1906_03065_gb300 import workloads as W

CS2 = 1.0 / 3.0


def _nb(a, c, shape):
    """a(x + c) on a periodic grid; a is flat, shape is (ny, nx) or (nz, ny, nx)."""
    A = a.reshape(shape)
    if len(shape) == 2:
        return np.roll(A, shift=(-c[1], -c[0]), axis=(0, 1)).ravel()
    return np.roll(A, shift=(-c[2], -c[1], -c[0]), axis=(0, 1, 2)).ravel()


def _free_energy(o, rho, phi, psi, I, p):
    """Discrete free energy without the ideal-gas part: bulk Landau terms,
    coupling term and gradient terms written as (3/2) sum_i w_i (dC)^2 (the
    lattice form of |grad C|^2 / 2 for these velocity sets)."""
    c, w = o.lattice()
    C1, C2, C3 = 0.5 * (rho + phi - psi), 0.5 * (rho - phi - psi), psi
    k = (p.kappa1, p.kappa2, p.kappa3)
    E = 0.0
    for km, Cm in zip(k, (C1, C2, C3)):
        E += (km / 2 * Cm ** 2 * (1 - Cm) ** 2).sum()
        g = sum(w[i] * (_nb(Cm, c[i], o.shape) - Cm) ** 2 for i in range(1, len(w)))
        E += p.alpha ** 2 * km * 1.5 * g.sum()
    E += (p.kappa_c / 2 * (psi - I) ** 2).sum()
    return E


@pytest.mark.parametrize("dim", [2, 3])
def test_potentials_are_variational_derivatives(dim):
    if dim == 2:
        wl = W.small_2d(nx=12, ny=10)
    else:
        wl = W.small_3d(nx=8, ny=7, nz=6, wall=0)
    p = wl.params
    p.alpha = 1.3
    wl.membranes = []
    o = oracle.Oracle(wl, init=False)
    rng = np.random.default_rng(7)
    N = o.N
    rho = 1 + 0.05 * rng.standard_normal(N)
    phi = rng.uniform(-1, 1, N)
    psi = rng.uniform(0, 1, N)
    I = rng.uniform(0, 1, N)
    mur, mup, mus = o.potentials(rho, phi, psi, I)
    h = 1e-6
    for cell in (0, 5, N // 2, N - 1):
        for arr, mu in ((rho, mur), (phi, mup), (psi, mus)):
            a0 = arr[cell]
            arr[cell] = a0 + h
            Ep = _free_energy(o, rho, phi, psi, I, p)
            arr[cell] = a0 - h
            Em = _free_energy(o, rho, phi, psi, I, p)
            arr[cell] = a0
            fd = (Ep - Em) / (2 * h)
            assert abs(fd - mu[cell]) < 1e-8 * max(1.0, abs(mu[cell])), (cell, fd, mu[cell])


def test_bulk_minima_and_rest_state_are_stationary():
    for (c1, c2, c3) in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        wl = W.small_2d(nx=8, ny=6)
        wl.membranes = []
        wl.params.kappa_c = 0.0
        o = oracle.Oracle(wl, init=False)
        N = o.N
        Cf = np.stack([np.full(N, c1, float), np.full(N, c2, float), np.full(N, c3, float)])
        o.init(Cf, np.zeros((3, N)))
        P0 = o.pops()
        o.step(3)
        # stationary up to the rounding of rho = sum_i f_i (1 +- 1 ulp)
        assert np.abs(o.pops() - P0).max() < 1e-15
        for name in ("mu_rho", "mu_phi", "mu_psi"):
            assert np.abs(o.field(name)).max() < 1e-16


def _unstream(P, c, shape):
    """Post-collision populations from streamed ones: f*_i(y) = f_i(y + c_i)."""
    return np.stack([_nb(P[i], c[i], shape) for i in range(len(c))])


@pytest.mark.parametrize("dim,tau", [(2, 1.0), (2, 0.8), (3, 1.0)])
def test_collision_moments(dim, tau):
    if dim == 2:
        wl = W.small_2d(nx=24, ny=22, nodes=30, radius=5.0, centre=(11.5, 10.7))
    else:
        wl = W.small_3d(nx=14, ny=13, nz=12, level=1, radius=3.5, centre=(7.1, 6.4, 5.8), wall=0)
    p = wl.params
    p.tau = p.tau_phi = p.tau_psi = tau
    o = oracle.Oracle(wl, init=False)
    C0, u0 = W.random_fields(p, seed=3)
    o.init(C0, u0)
    # random non-equilibrium part, with zero mass / momentum change
    rng = np.random.default_rng(9)
    P = o.pops()
    c, w = o.lattice()
    P = P + 1e-3 * rng.standard_normal(P.shape) * w[None, :, None]
    o.set_pops(P)
    rho, phi, psi = P[0].sum(0), P[1].sum(0), P[2].sum(0)
    j = np.einsum("ia,in->an", c, P[0])
    G1 = np.einsum("ia,in->an", c, P[1])
    o.step(1)
    S = _unstream(o.pops().reshape(3, len(c), -1)[0], c, o.shape)
    Sg = _unstream(o.pops()[1], c, o.shape)
    Sh = _unstream(o.pops()[2], c, o.shape)
    F = np.stack([o.field("Fx"), o.field("Fy"), o.field("Fz")])
    assert np.abs(S.sum(0) - rho).max() < 1e-13
    assert np.abs(Sg.sum(0) - phi).max() < 1e-13
    assert np.abs(Sh.sum(0) - psi).max() < 1e-13
    # momentum changes by exactly the force (exact-difference forcing)
    assert np.abs(np.einsum("ia,in->an", c, S) - (j + F)).max() < 1e-13
    u = j / rho
    v = u + 0.5 * F / rho
    d = np.eye(3)
    if tau == 1.0:
        # tau = 1: f* = f^eq(rho, u + du), g* = g^eq(phi, v): second moments
        ud = u + F / rho
        M2 = np.einsum("ia,ib,in->abn", c, c, S)
        ref = rho * CS2 * d[:, :, None] + rho * ud[:, None] * ud[None, :]
        if dim == 2:
            M2, ref = M2[:2, :2], ref[:2, :2]
        assert np.abs(M2 - ref).max() < 1e-13
        for Sx, a, mu, G in ((Sg, phi, o.field("mu_phi"), p.gamma_phi),
                             (Sh, psi, o.field("mu_psi"), p.gamma_psi)):
            assert np.abs(np.einsum("ia,in->an", c, Sx) - a * v).max() < 1e-13
            M2 = np.einsum("ia,ib,in->abn", c, c, Sx)
            ref = G * mu * d[:, :, None] + a * v[:, None] * v[None, :]
            if dim == 2:
                M2, ref = M2[:2, :2], ref[:2, :2]
            assert np.abs(M2 - ref).max() < 1e-13
    else:
        Gp = np.einsum("ia,in->an", c, Sg)
        ref = (1 - 1 / tau) * G1 + (1 / tau) * phi * v
        assert np.abs(Gp - ref).max() < 1e-13


@pytest.mark.parametrize("dim,tau", [(2, 1.0), (2, 0.8), (3, 0.7)])
def test_guo_forcing_collision_moments(dim, tau):
    """Guo forcing (Guo, Zheng and Shi 2002): mass is conserved, momentum
    changes by exactly F, and the second moment relaxes towards the
    equilibrium at v = (j + F/2)/rho with the source's (1 - 1/(2 tau))
    (v F + F v) -- the published moments of the scheme."""
    if dim == 2:
        wl = W.small_2d(nx=24, ny=22, nodes=30, radius=5.0, centre=(11.5, 10.7))
    else:
        wl = W.small_3d(nx=14, ny=13, nz=12, level=1, radius=3.5, centre=(7.1, 6.4, 5.8), wall=0)
    p = wl.params
    p.tau = p.tau_phi = p.tau_psi = tau
    p.forcing = "guo"
    o = oracle.Oracle(wl, init=False)
    C0, u0 = W.random_fields(p, seed=3)
    o.init(C0, u0)
    rng = np.random.default_rng(11)
    P = o.pops()
    c, w = o.lattice()
    P = P + 1e-3 * rng.standard_normal(P.shape) * w[None, :, None]
    o.set_pops(P)
    rho = P[0].sum(0)
    j = np.einsum("ia,in->an", c, P[0])
    Pi = np.einsum("ia,ib,in->abn", c, c, P[0])
    o.step(1)
    S = _unstream(o.pops().reshape(3, len(c), -1)[0], c, o.shape)
    F = np.stack([o.field("Fx"), o.field("Fy"), o.field("Fz")])
    assert np.abs(F).max() > 1e-6  # the forces are not trivial
    assert np.abs(S.sum(0) - rho).max() < 1e-13
    assert np.abs(np.einsum("ia,in->an", c, S) - (j + F)).max() < 1e-13
    v = (j + 0.5 * F) / rho
    d = np.eye(3)
    eq = rho * CS2 * d[:, :, None] + rho * v[:, None] * v[None, :]
    src = (1 - 0.5 / tau) * (v[:, None] * F[None, :] + F[:, None] * v[None, :])
    ref = (1 - 1 / tau) * Pi + eq / tau + src
    M2 = np.einsum("ia,ib,in->abn", c, c, S)
    if dim == 2:
        M2, ref = M2[:2, :2], ref[:2, :2]
    assert np.abs(M2 - ref).max() < 1e-13


def test_mass_conservation_with_capsule_and_walls():
    wl = W.small_3d(nx=20, ny=18, nz=16, level=2, radius=5.0, centre=(10.2, 9.1, 8.3))
    o = oracle.Oracle(wl)
    m0 = o.masses()
    o.step(12)
    m1 = o.masses()
    assert np.abs(m1 - m0).max() <= 1e-12 * np.abs(m0).max()
    wl2 = W.capsule_2d()
    o2 = oracle.Oracle(wl2)
    m0 = o2.masses()
    o2.step(50)
    assert np.abs(o2.masses() - m0).max() <= 1e-12 * np.abs(m0).max()


def test_integer_shift_equivariance():
    """Shifting the initial fields and the capsule by an integer vector shifts
    the whole evolution (periodic lattice, eqs. LBE, Spreading, Interpolation)."""
    wl = W.small_2d()
    o = oracle.Oracle(wl)
    C0 = np.stack([o.field(n).reshape(o.shape) for n in ("C1", "C2", "C3")])
    a = oracle.Oracle(wl, init=False)
    a.init(C0.reshape(3, -1), None)
    a.step(25)
    wl2 = W.small_2d(centre=(20.3 + 7, 17.6 + 5))
    b = oracle.Oracle(wl2, init=False)
    b.init(np.roll(C0, (5, 7), axis=(1, 2)).reshape(3, -1), None)
    b.step(25)
    for name in ("phi", "psi", "ux", "uy"):
        fa = a.field(name).reshape(o.shape)
        fb = b.field(name).reshape(o.shape)
        assert np.abs(np.roll(fa, (5, 7), axis=(0, 1)) - fb).max() < 1e-10, name
    assert np.abs(b.nodes(0) - a.nodes(0) - np.array([7, 5, 0])).max() < 1e-10


def _droplet(n, R, u0, kappa=(0.01, 0.01, 0.01), alpha=1.0):
    wl = W.small_2d(nx=n, ny=n)
    wl.membranes = []
    p = wl.params
    p.kappa1, p.kappa2, p.kappa3 = kappa
    p.kappa_c = 0.0
    p.alpha = alpha
    p.gamma_phi = p.gamma_psi = 1.0
    o = oracle.Oracle(wl, init=False)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r = np.hypot(x - n / 2 + 0.5, y - n / 2 + 0.5).ravel()
    C3 = 0.5 * (1 - np.tanh((r - R) / (2 * alpha)))
    Cf = np.stack([1 - C3, np.zeros_like(C3), C3])
    u = np.zeros((3, o.N))
    u[0] += u0[0]
    u[1] += u0[1]
    o.init(Cf, u)
    return o, p


def _centroid_x(p):
    n = p.shape[1]
    ang = 2 * np.pi * np.arange(n) / n
    col = p.sum(0)
    return np.arctan2((col * np.sin(ang)).sum(), (col * np.cos(ang)).sum()) * n / (2 * np.pi)


def _gyration(p, cx):
    n = p.shape[0]
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    dx = (xx - cx + n / 2) % n - n / 2
    dy = yy - (p * yy).sum() / p.sum()
    return np.sqrt((dx ** 2 * p).sum() / p.sum()), np.sqrt((dy ** 2 * p).sum() / p.sum())


def test_galilean_translation_of_droplet():
    """A droplet in a uniformly moving fluid (U_x0 as in Sec. 4.1) travels at
    U and relaxes to the same shape as a resting one: centroid displacement
    U t and equal radii of gyration along and across the motion."""
    n, steps, U = 40, 160, 0.05
    a, _ = _droplet(n, 9.0, (0.0, 0.0))
    b, _ = _droplet(n, 9.0, (U, 0.0))
    a.step(steps)
    b.step(steps)
    pa = a.field("psi").reshape(n, n)
    pb = b.field("psi").reshape(n, n)
    ca, cb = _centroid_x(pa), _centroid_x(pb)
    disp = (cb - ca + n / 2) % n - n / 2
    assert abs(disp - U * steps) < 0.1, disp
    ga, gb = _gyration(pa, ca), _gyration(pb, cb)
    assert abs(gb[0] / ga[0] - 1) < 1e-3 and abs(gb[1] / ga[1] - 1) < 1e-3, (ga, gb)
    assert abs(pb.sum() / pa.sum() - 1) < 1e-12


def _pressure(o, p, cell):
    """Bulk pressure p_b = rho cs^2 + sum_m C_m df/dC_m - f with
    f = sum_m kappa_m/2 C_m^2 (1 - C_m)^2 (eqs. PressureV2, BulkPres)."""
    C = np.array([o.field("C1")[cell], o.field("C2")[cell], o.field("C3")[cell]])
    k = np.array([p.kappa1, p.kappa2, p.kappa3])
    f = (k / 2 * C ** 2 * (1 - C) ** 2).sum()
    dfdC = k * C * (1 - C) * (1 - 2 * C)
    return o.field("rho")[cell] * CS2 + (C * dfdC).sum() - f


@pytest.mark.slow
def test_laplace_law():
    n = 48
    res = []
    for R in (10.0, 14.0):
        o, p = _droplet(n, R, (0.0, 0.0), kappa=(0.01, 0.01, 0.01), alpha=1.0)
        o.step(4000)
        psi = o.field("psi")
        Reff = math.sqrt(psi.sum() / math.pi)
        centre = (n // 2) * n + n // 2
        dp = _pressure(o, p, centre) - _pressure(o, p, 0)
        g13 = p.alpha * (p.kappa1 + p.kappa3) / 6
        res.append(dp / (g13 / Reff))
    for r in res:
        assert abs(r - 1) < 0.06, res


@pytest.mark.slow
@pytest.mark.parametrize("pair", [(1, 2), (1, 3), (2, 3)])
def test_flat_interface_profile_and_tension(pair):
    """Component m between y = 32 and 96 in a periodic 4x128 strip of
    component n, started on the profile (1 + tanh(d/(2 alpha)))/2 of eq.
    CmProfile: it stays there (the discrete equilibrium differs from the
    continuum one by O(1e-3)) and each interface carries the excess free
    energy gamma_mn = alpha (kappa_m + kappa_n)/6 of eq. SurfaceTension, for
    each of the three pairs (kappa = 0.01, 0.02, 0.015: three different
    tensions).  (The width itself relaxes on a slow Cahn-Hilliard time
    scale, so the start is the target profile.)"""
    m, n = pair
    ny, alpha = 128, 2.0
    wl = W.small_2d(nx=4, ny=ny)
    wl.membranes = []
    p = wl.params
    p.alpha = alpha
    p.kappa1, p.kappa2, p.kappa3, p.kappa_c = 0.01, 0.02, 0.015, 0.0
    p.gamma_phi = p.gamma_psi = 1.0
    o = oracle.Oracle(wl, init=False)
    y = np.repeat(np.arange(ny), 4).astype(float)
    s = 0.5 * (np.tanh((y - 32) / (2 * alpha)) - np.tanh((y - 96) / (2 * alpha)))
    Cf = np.zeros((3, o.N))
    Cf[m - 1] = s
    Cf[n - 1] = 1 - s
    o.init(Cf, np.zeros((3, o.N)))
    o.step(3000)
    Cm = o.field(f"C{m}").reshape(ny, 4)[:, 0]
    # interface position from the half crossing near y = 32
    k = np.where((Cm[:-1] < 0.5) & (Cm[1:] >= 0.5))[0][0]
    y0 = k + (0.5 - Cm[k]) / (Cm[k + 1] - Cm[k])
    yy = np.arange(16, 48)
    prof = 0.5 * (1 + np.tanh((yy - y0) / (2 * alpha)))
    assert np.abs(Cm[16:48] - prof).max() < 5e-3
    # excess free energy per interface (bulk + gradient, per unit length)
    C = [o.field(nm).reshape(ny, 4)[:, 0] for nm in ("C1", "C2", "C3")]
    k3 = (p.kappa1, p.kappa2, p.kappa3)
    e = 0.0
    for km, Ck in zip(k3, C):
        dC = 0.5 * (np.roll(Ck, -1) - np.roll(Ck, 1))
        e += (km / 2 * Ck ** 2 * (1 - Ck) ** 2 + alpha ** 2 * km / 2 * dC ** 2).sum()
    gam = e / 2
    ref = alpha * (k3[m - 1] + k3[n - 1]) / 6
    assert abs(gam / ref - 1) < 0.02, (pair, gam, ref)


def _circle_fit(x, y):
    """Least-squares circle through points (algebraic fit): centre, radius."""
    A = np.stack([x, y, np.ones_like(x)], 1)
    c, *_ = np.linalg.lstsq(A, x ** 2 + y ** 2, rcond=None)
    cx, cy = c[0] / 2, c[1] / 2
    return cx, cy, math.sqrt(c[2] + cx ** 2 + cy ** 2)


def _contour(F, lev=0.5):
    """Points of the level set F = lev by linear interpolation along rows
    and columns of a 2D array F[y, x]."""
    ny, nx = F.shape
    pts = []
    for j in range(ny):
        r = F[j]
        for i in range(nx - 1):
            if (r[i] - lev) * (r[i + 1] - lev) < 0:
                pts.append((i + (lev - r[i]) / (r[i + 1] - r[i]), j))
    for i in range(nx):
        c = F[:, i]
        for j in range(ny - 1):
            if (c[j] - lev) * (c[j + 1] - lev) < 0:
                pts.append((i, j + (lev - c[j]) / (c[j + 1] - c[j])))
    return np.array(pts)


def _relaxed_lens(nx, ny, R, kappa, steps, alpha=1.0):
    """A C3 disc of radius R centred on a flat C1 (above) / C2 (below)
    interface between walls, no membrane, relaxed for ``steps``; returns the
    two lens angles at the triple points, measured from circles fitted to
    the C3 = 1/2 contour above and below the interface band: beta1 between
    the C1/C2 interface and the C1/C3 arc, beta2 with the C2/C3 arc."""
    wl = W.small_2d(nx=nx, ny=ny)
    wl.membranes = []
    p = wl.params
    p.wall_last = 1
    p.kappa1, p.kappa2, p.kappa3 = kappa
    p.kappa_c, p.alpha = 0.0, alpha
    p.gamma_phi = p.gamma_psi = 1.0
    o = oracle.Oracle(wl, init=False)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    y0 = ny / 2 - 0.5
    C3 = 0.5 * (1 - np.tanh((np.hypot(x - nx / 2 + 0.5, y - y0) - R) / (2 * alpha)))
    s = 0.5 * (1 + np.tanh((y - y0) / (2 * alpha)))
    o.init(np.stack([(1 - C3) * s, (1 - C3) * (1 - s), C3]).reshape(3, -1), np.zeros((3, o.N)))
    o.step(steps)
    psi = o.field("psi").reshape(ny, nx)
    phi = o.field("phi").reshape(ny, nx)
    yi = []  # far-field height of the C1/C2 interface (phi = 0)
    for i in list(range(6)) + list(range(nx - 6, nx)):
        c = phi[:, i]
        j = np.where((c[:-1] < 0) & (c[1:] >= 0))[0][0]
        yi.append(j - c[j] / (c[j + 1] - c[j]))
    yint = float(np.mean(yi))
    P = _contour(psi)
    up, lo = P[P[:, 1] > yint + 2 * alpha], P[P[:, 1] < yint - 2 * alpha]
    (x1, y1, r1), (x2, y2, r2) = _circle_fit(up[:, 0], up[:, 1]), _circle_fit(lo[:, 0], lo[:, 1])
    # the triple points: intersections of the two circles
    d = math.hypot(x2 - x1, y2 - y1)
    a1 = (r1 ** 2 - r2 ** 2 + d ** 2) / (2 * d)
    hh = math.sqrt(r1 ** 2 - a1 ** 2)
    ym = y1 + a1 * (y2 - y1) / d
    half = hh  # the circles' centres lie on one vertical line (mirror symmetry)
    b1 = math.degrees(math.atan2(half, ym - y1))
    b2 = math.degrees(math.atan2(half, y2 - ym))
    return b1, b2, ym - yint


@pytest.mark.slow
def test_neumann_triangle_of_a_ternary_lens():
    """A pure ternary lens (no membrane) relaxes to the angles of the
    Neumann triangle of its three tensions (eq. SurfaceTension): at a triple
    point gamma_12 t_12 + gamma_13 t_13 + gamma_23 t_23 = 0, i.e. with the
    C1/C2 interface flat, cos beta1 = (g12^2 + g13^2 - g23^2)/(2 g12 g13) and
    cos beta2 = (g12^2 + g23^2 - g13^2)/(2 g12 g23).  kappa = (0.03, 0.018,
    0.024) gives beta1 = 48.19 and beta2 = 73.40 degrees.  The diffuse
    interfaces (width ~ 4 alpha) shift the measured angles by a first-order
    amount in alpha/R; measured: +0.62 / +1.01 degrees at R = 10 and +0.23 /
    +0.63 at R = 14, so the tolerance is 1.5 degrees with the error required
    to shrink under that refinement.  Swapping two tensions moves an angle
    by 25 degrees."""
    kap = (0.03, 0.018, 0.024)
    g12, g13, g23 = kap[0] + kap[1], kap[0] + kap[2], kap[1] + kap[2]  # times alpha/6
    e1 = math.degrees(math.acos((g12 ** 2 + g13 ** 2 - g23 ** 2) / (2 * g12 * g13)))
    e2 = math.degrees(math.acos((g12 ** 2 + g23 ** 2 - g13 ** 2) / (2 * g12 * g23)))
    errs = []
    for nx, ny, R, steps in ((64, 48, 10.0, 12000), (96, 64, 14.0, 16000)):
        b1, b2, dy = _relaxed_lens(nx, ny, R, kap, steps)
        errs.append((b1 - e1, b2 - e2))
        assert abs(b1 - e1) < 1.5 and abs(b2 - e2) < 1.5, (R, b1, b2, e1, e2)
        assert abs(dy) < 0.5  # the triple line lies on the far-field interface
    assert sum(map(abs, errs[1])) < sum(map(abs, errs[0])), errs
