"""Pins of the oracle's equilibrium-quality measures (no GPU).

* capsule area and volume: the shoelace area of a regular polygon, the area
  and volume of the regular icosahedron (closed forms), convergence of the
  subdivided icosphere to 4 pi R^2 and 4 pi R^3 / 3, invariance under
  translation and the sign of the orientation;
* the contact angle of a membrane with the C1/C2 interface phi = 0: a
  sphere whose centre lies a distance h above a flat (or tilted) tanh
  interface meets it at the angle arccos(-h/R) between the interface normal
  (into C1) and the outward membrane normal, and a ring in 2D likewise.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1906_03065_gb300 import workloads as W


def test_regular_polygon_area_and_orientation():
    for n, R in ((76, 12.0), (9, 3.0), (200, 30.0)):
        wl = W.small_2d(nodes=n, radius=R, centre=(20.3, 17.6))
        o = oracle.Oracle(wl, init=False)
        X = wl.membranes[0].X
        A, V = o.capsule_measures(0, X)
        assert abs(A - 0.5 * n * R * R * math.sin(2 * math.pi / n)) < 1e-10 * R * R
        assert V == 0.0
        # translation invariance and the sign of a clockwise ring
        A2, _ = o.capsule_measures(0, X + np.array([7.25, -3.5, 0.0]))
        assert abs(A2 - A) < 1e-10 * R * R
        A3, _ = o.capsule_measures(0, X * np.array([1.0, -1.0, 1.0]))
        assert abs(A3 + A) < 1e-10 * R * R


def test_icosahedron_area_and_volume_closed_forms():
    R = 5.0
    wl = W.small_3d(nx=24, ny=24, nz=24, level=0, radius=R, centre=(12.1, 11.8, 12.3))
    o = oracle.Oracle(wl, init=False)
    X = wl.membranes[0].X
    a = 4 * R / math.sqrt(10 + 2 * math.sqrt(5))  # edge of the icosahedron of circumradius R
    A, V = o.capsule_measures(0, X)
    assert abs(A - 5 * math.sqrt(3) * a * a) < 1e-10 * A
    assert abs(V - 5 / 12 * (3 + math.sqrt(5)) * a ** 3) < 1e-10 * V
    # translation does not change the enclosed volume; reversed triangles flip it
    _, V2 = o.capsule_measures(0, X + np.array([100.0, -40.0, 7.0]))
    assert abs(V2 - V) < 1e-9 * V
    wl.membranes[0].elems = wl.membranes[0].elems[:, ::-1].copy()
    o2 = oracle.Oracle(wl, init=False)
    _, V3 = o2.capsule_measures(0, X)
    assert abs(V3 + V) < 1e-10 * V


def test_icosphere_measures_converge_to_the_sphere():
    R = 10.0
    err_a, err_v = [], []
    for level in (2, 3, 4):
        wl = W.small_3d(nx=32, ny=32, nz=32, level=level, radius=R, centre=(16.2, 15.9, 16.1))
        o = oracle.Oracle(wl, init=False)
        A, V = o.capsule_measures(0, wl.membranes[0].X)
        err_a.append(abs(A / (4 * math.pi * R * R) - 1))
        err_v.append(abs(V / (4 / 3 * math.pi * R ** 3) - 1))
    # second order in the edge length: each level halves it
    for e in (err_a, err_v):
        assert e[1] < e[0] / 3.2 and e[2] < e[1] / 3.2, e
    assert err_a[2] < 2e-3 and err_v[2] < 3e-3


def _phi_plane(n, normal, p0, alpha):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    d = (x - p0[0]) * normal[0] + (y - p0[1]) * normal[1] + (z - p0[2]) * normal[2]
    return np.tanh(d / (2 * alpha)).ravel()


@pytest.mark.parametrize("h", [-4.0, 0.0, 2.5, 6.0])
def test_sphere_on_flat_interface_contact_angle(h):
    n, R = 48, 20.0
    c = (n / 2 + 0.31, n / 2 - 0.17, n / 2 + h)
    wl = W.small_3d(nx=n, ny=n, nz=n, level=4, radius=R, centre=c)
    o = oracle.Oracle(wl, init=False)
    phi = _phi_plane(n, (0.0, 0.0, 1.0), (0.0, 0.0, n / 2), 2.0)
    (mean, lo, hi), cnt = o.contact_angle(0, wl.membranes[0].X, phi)
    assert cnt >= 32
    # the error of the polyhedral surface and its interpolated normals
    assert abs(mean - math.degrees(math.acos(-h / R))) < 0.1, (mean, h)
    assert hi - lo < 1.0


def test_sphere_on_tilted_interface_contact_angle():
    """The interface normal is the lattice gradient of phi, not a fixed axis:
    a tilted plane gives the same arccos(-d/R) with d the signed distance of
    the centre along the plane's normal."""
    n, R = 48, 20.0
    nrm = np.array([0.3, -0.2, 1.0])
    nrm /= np.linalg.norm(nrm)
    c = np.array([n / 2 + 0.2, n / 2 - 0.3, n / 2 + 1.7])
    p0 = np.array([n / 2, n / 2, n / 2 - 1.0])
    wl = W.small_3d(nx=n, ny=n, nz=n, level=4, radius=R, centre=tuple(c), wall=0)
    o = oracle.Oracle(wl, init=False)
    phi = _phi_plane(n, nrm, p0, 2.0)
    (mean, _, _), cnt = o.contact_angle(0, wl.membranes[0].X, phi)
    d = float(np.dot(c - p0, nrm))
    assert cnt > 100
    assert abs(mean - math.degrees(math.acos(-d / R))) < 0.1, (mean, d)


@pytest.mark.parametrize("h", [-3.0, 0.0, 5.0])
def test_ring_on_flat_interface_contact_angle(h):
    n, R = 64, 12.0
    wl = W.small_2d(nx=n, ny=n, nodes=76, radius=R, centre=(32.3, 32.0 + h))
    o = oracle.Oracle(wl, init=False)
    y = np.repeat(np.arange(n), n).astype(float)
    phi = np.tanh((y - 32.0) / 2.0)
    (mean, lo, hi), cnt = o.contact_angle(0, wl.membranes[0].X, phi)
    assert cnt == 2
    assert abs(mean - math.degrees(math.acos(-h / R))) < 0.1, (mean, h)
    assert abs(lo - hi) < 0.2


def test_no_contact_when_the_membrane_misses_the_interface():
    n = 32
    wl = W.small_3d(nx=n, ny=n, nz=n, level=2, radius=5.0, centre=(16.1, 15.8, 8.0))
    o = oracle.Oracle(wl, init=False)
    phi = _phi_plane(n, (0.0, 0.0, 1.0), (0.0, 0.0, 24.0), 1.0)
    out, cnt = o.contact_angle(0, wl.membranes[0].X, phi)
    assert cnt == 0 and np.isnan(out).all()
