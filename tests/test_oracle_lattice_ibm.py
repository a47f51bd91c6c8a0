"""Pins of the oracle's lattice, Peskin kernel, spreading/interpolation and
membrane profile against facts the paper or mathematics fix (no GPU)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1906_03065_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_d2q9_matches_printed_table():
    g = json.load(open(os.path.join(GOLD, "d2q9_table.json")))
    o = oracle.Oracle(W.small_2d(), init=False)
    c, w = o.lattice()
    assert list(c[:, 0]) == g["cx"]
    assert list(c[:, 1]) == g["cy"]
    assert np.allclose(w, [float(Fraction(x)) for x in g["w"]], rtol=0, atol=1e-16)


def test_d3q19_isotropy():
    """Weights and velocities of D3Q19: sum w = 1, odd moments vanish,
    sum w c_a c_b = cs^2 delta, 4th moment = cs^4 (dd + dd + dd)."""
    o = oracle.Oracle(W.small_3d(), init=False)
    c, w = o.lattice()
    assert c.shape == (19, 3)
    assert abs(w.sum() - 1) < 1e-15
    cs2 = 1.0 / 3.0
    d = np.eye(3)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), cs2 * d, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-15)


@pytest.mark.parametrize("r", [0.0, 0.13, 0.5, 0.77, 0.999])
def test_peskin_moment_identities(r):
    """Peskin's 4-point kernel (eq. DiscreteDirac): partition of unity, zero
    first moment and sum of squares 3/8 for every shift r."""
    js = np.arange(-3, 4)
    v = np.array([oracle.peskin(r - j) for j in js])
    assert abs(v.sum() - 1) < 1e-14
    assert abs(((r - js) * v).sum()) < 1e-14
    assert abs((v ** 2).sum() - 3.0 / 8.0) < 1e-14
    assert oracle.peskin(2.0) == 0.0 and oracle.peskin(-2.5) == 0.0


def test_spread_conserves_total_and_interp_is_exact_for_linear():
    wl = W.small_3d(nx=24, ny=22, nz=20, level=1, radius=5.0, centre=(11.3, 10.7, 9.6))
    o = oracle.Oracle(wl, init=False)
    X = wl.membranes[0].X
    rng = np.random.default_rng(3)
    F = rng.normal(size=X.shape)
    fib = o.spread(X, F)
    assert np.allclose(fib.sum(axis=1), F.sum(axis=0), rtol=0, atol=1e-12)
    # interpolation of a linear field (inside the domain, no wrap) is exact
    z, y, x = np.meshgrid(np.arange(20), np.arange(22), np.arange(24), indexing="ij")
    field = np.stack([0.3 + 0.01 * x - 0.02 * y, 0.05 * z, -0.1 + 0.002 * x + 0.003 * z])
    U = o.interp(X, field.reshape(3, -1))
    ex = np.stack([0.3 + 0.01 * X[:, 0] - 0.02 * X[:, 1], 0.05 * X[:, 2],
                   -0.1 + 0.002 * X[:, 0] + 0.003 * X[:, 2]], axis=1)
    assert np.abs(U - ex).max() < 1e-12


def _ring_brute(X, pts):
    """Independent brute force: distance to the polyline and even-odd ray
    casting for the inside test."""
    A = X[:, :2]
    B = np.roll(A, -1, axis=0)
    d = np.full(len(pts), np.inf)
    inside = np.zeros(len(pts), dtype=bool)
    for a, b in zip(A, B):
        ab = b - a
        t = np.clip(((pts - a) @ ab) / (ab @ ab), 0, 1)
        P = a + t[:, None] * ab
        d = np.minimum(d, np.linalg.norm(pts - P, axis=1))
        cond = (a[1] > pts[:, 1]) != (b[1] > pts[:, 1])
        xint = a[0] + (pts[:, 1] - a[1]) * ab[0] / np.where(ab[1] == 0, 1, ab[1])
        inside ^= cond & (pts[:, 0] < xint)
    return np.where(inside, d, -d)


def test_iprofile_2d_matches_brute_force():
    wl = W.small_2d(nx=30, ny=28, nodes=40, radius=7.0, centre=(14.4, 13.3))
    m = W.jitter_nodes(wl.membranes[0], 0.3, seed=5)
    wl.membranes[0] = m
    o = oracle.Oracle(wl, init=False)
    I, d, nb = o.iprofile(m.X)
    y, x = np.meshgrid(np.arange(28), np.arange(30), indexing="ij")
    pts = np.stack([x.ravel(), y.ravel()], axis=1).astype(float)
    ref = np.clip(_ring_brute(m.X, pts), -wl.params.dc, wl.params.dc)
    assert np.abs(d - ref).max() < 1e-12
    Iref = 0.5 * (1 + np.tanh(ref / (2 * wl.params.alpha)))
    assert np.abs(I - Iref).max() < 1e-14
    assert nb == int((np.abs(ref) < wl.params.dc).sum())


def test_iprofile_3d_matches_sampled_surface():
    """Distance to a jittered icosphere versus a dense barycentric sampling of
    its triangles (an upper bound converging to the distance) and a ray
    parity inside test."""
    wl = W.small_3d(nx=16, ny=16, nz=16, level=1, radius=4.5, centre=(7.6, 8.2, 7.9))
    m = W.jitter_nodes(wl.membranes[0], 0.15, seed=2)
    wl.membranes[0] = m
    o = oracle.Oracle(wl, init=False)
    I, d, nb = o.iprofile(m.X)
    n = 24
    a, b = np.meshgrid(np.linspace(0, 1, n + 1), np.linspace(0, 1, n + 1), indexing="ij")
    keep = a + b <= 1 + 1e-12
    a, b = a[keep], b[keep]
    T = m.elems
    P0, P1, P2 = m.X[T[:, 0]], m.X[T[:, 1]], m.X[T[:, 2]]
    S = (P0[:, None, :] * (1 - a - b)[None, :, None] + P1[:, None, :] * a[None, :, None]
         + P2[:, None, :] * b[None, :, None]).reshape(-1, 3)
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(float)
    # periodic in x and y (walls in z): all neighbouring images
    shifts = [np.array([i * 16.0, j * 16.0, 0.0]) for i in (-1, 0, 1) for j in (-1, 0, 1)]
    SS = np.concatenate([S + sh for sh in shifts])
    dmin = np.array([np.sqrt(((SS - p) ** 2).sum(1)).min() for p in pts])
    # ray parity along a generic direction (Moller-Trumbore)
    dirv = np.array([0.5361, 0.3377, 0.7738])
    e1, e2 = P1 - P0, P2 - P0
    inside = np.zeros(len(pts), dtype=bool)
    for k, p in enumerate(pts):
        for sh in shifts:
            h = np.cross(dirv, e2)
            det = (e1 * h).sum(1)
            s = p - (P0 + sh)
            u = (s * h).sum(1) / det
            q = np.cross(s, e1)
            v = (q @ dirv) / det
            t = (q * e2).sum(1) / det
            hit = (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
            inside[k] |= hit.sum() % 2 == 1
    ref = np.where(inside, dmin, -dmin)
    dc = wl.params.dc
    refc = np.clip(ref, -dc, dc)
    # sampled distance is an upper bound within the sampling resolution
    err = np.abs(np.abs(d) - np.abs(refc))
    assert err.max() < 0.05
    far = np.abs(refc) > 0.1
    assert np.all(np.sign(d[far]) == np.sign(refc[far]))


def _fd_check(fun_E, X, F, idx, h=1e-6, dims=3):
    for (l, k) in idx:
        if k >= dims:
            continue
        Xp = X.copy(); Xp[l, k] += h
        Xm = X.copy(); Xm[l, k] -= h
        g = (fun_E(Xp) - fun_E(Xm)) / (2 * h)
        assert abs(-g - F[l, k]) <= 1e-6 * max(1e-3, np.abs(F).max()), (l, k, -g, F[l, k])


def test_coupling_force_is_minus_gradient_2d():
    wl = W.small_2d(nx=32, ny=30, nodes=44, radius=7.0, centre=(15.4, 14.2))
    m = W.jitter_nodes(wl.membranes[0], 0.25, seed=11)
    wl.membranes[0] = m
    o = oracle.Oracle(wl, init=False)
    rng = np.random.default_rng(0)
    psi = rng.uniform(0, 1, o.N)
    E, F = o.coupling(psi, m.X)
    fun = lambda X: o.coupling(psi, X, want_force=False)[0]
    idx = [(l, k) for l in (0, 7, 19, 30) for k in (0, 1)]
    _fd_check(fun, m.X.copy(), F, idx, dims=2)


def test_coupling_force_is_minus_gradient_3d():
    wl = W.small_3d(nx=18, ny=18, nz=18, level=1, radius=4.5, centre=(8.6, 9.2, 8.9))
    m = W.jitter_nodes(wl.membranes[0], 0.15, seed=4)
    wl.membranes[0] = m
    o = oracle.Oracle(wl, init=False)
    rng = np.random.default_rng(1)
    psi = rng.uniform(0, 1, o.N)
    E, F = o.coupling(psi, m.X)
    fun = lambda X: o.coupling(psi, X, want_force=False)[0]
    idx = [(l, k) for l in (0, 5, 17, 33) for k in (0, 1, 2)]
    _fd_check(fun, m.X.copy(), F, idx, dims=3)


def test_tension_ratio_fixture():
    g = json.load(open(os.path.join(GOLD, "tension_ratios.json")))
    for c in g["cases"]:
        k1, k2, k3 = c["kappa"]
        gam = {"g12": k1 + k2, "g13": k1 + k3, "g23": k2 + k3}  # alpha/6 cancels
        num, den = c["ratio"].split("/")
        assert abs(gam[num] / gam[den] - c["printed"]) <= c["tol"], c["what"]
