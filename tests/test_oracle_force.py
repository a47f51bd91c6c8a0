"""Pins of the oracle's free-energy force (no GPU).

* The lattice gradient and Laplacian (the step's isotropic stencils) equal
  the analytic derivatives of smooth periodic fields to second order in the
  wavenumber: a wrong prefactor (for instance a missing or doubled 1/cs^2)
  fails at once.
* The bulk pressure p_b of App. A obeys the Gibbs-Duhem relation
  dp_b = rho dmu_rho + phi dmu_phi + psi dmu_psi of the bulk free energy of
  eq. LandauFE (the printed polynomial needs one more psi^2 term for this).
* The force of the step (potential form, eq. ForceFE through eq. GradPT)
  equals the literal first line of eq. ForceFE, grad(rho cs^2) - div p -
  psi grad(kappa_c (psi - I)) with the explicit pressure tensor of App. A,
  up to the second-order discretisation difference of the two forms: the
  difference falls by about 4 when the fields are resolved on twice as many
  lattice nodes.  A wrong magnitude of the gradient stencil would scale the
  two forms differently (one gradient against up to three) and fail here
  as well.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1906_03065_gb300 import workloads as W

CS2 = 1.0 / 3.0


def _lattice3(n, wall=0):
    wl = W.small_3d(nx=n, ny=n, nz=n, wall=wall)
    wl.membranes = []
    return oracle.Oracle(wl, init=False), wl.params


def _coords(n):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return x.ravel().astype(float), y.ravel().astype(float), z.ravel().astype(float)


def _field(n, phase=0.0):
    """A smooth periodic field with its analytic gradient and Laplacian."""
    x, y, z = _coords(n)
    k = 2 * math.pi / n
    a = np.sin(k * x + phase) * np.cos(2 * k * y) + 0.5 * np.sin(k * (x + y + z))
    gx = k * np.cos(k * x + phase) * np.cos(2 * k * y) + 0.5 * k * np.cos(k * (x + y + z))
    gy = -2 * k * np.sin(k * x + phase) * np.sin(2 * k * y) + 0.5 * k * np.cos(k * (x + y + z))
    gz = 0.5 * k * np.cos(k * (x + y + z))
    L = -5 * k * k * np.sin(k * x + phase) * np.cos(2 * k * y) - 1.5 * k * k * np.sin(k * (x + y + z))
    return a, np.stack([gx, gy, gz]), L, k


def test_gradient_and_laplacian_stencils_are_second_order():
    errs = []
    for n in (16, 32):
        o, _ = _lattice3(n)
        a, g, L, k = _field(n, 0.3)
        eg = np.abs(o.grad_field(a) - g).max() / np.abs(g).max()
        eL = np.abs(o.lap_field(a) - L).max() / np.abs(L).max()
        errs.append((eg, eL))
    for q in range(2):
        assert errs[1][q] < errs[0][q] / 3.6, errs
    # (sin k - k)/k ~ -k^2/6 for the largest wavenumber of the field (2k)
    assert errs[1][0] < 0.03 and errs[1][1] < 0.03, errs


def test_gradient_stencil_in_2d_and_at_walls():
    n = 32
    wl = W.small_2d(nx=n, ny=n)
    wl.membranes = []
    o = oracle.Oracle(wl, init=False)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    k = 2 * math.pi / n
    a = np.sin(k * x + 2 * k * y).ravel()
    g = o.grad_field(a)
    # derivatives of sin(k x + 2k y): leading error |k|^2/6 relative (3.2 %)
    for d, kd in ((0, k), (1, 2 * k)):
        ref = (kd * np.cos(k * x + 2 * k * y)).ravel()
        assert np.abs(g[d] - ref).max() < 0.035 * kd, d
    assert np.abs(g[2]).max() == 0.0
    # walls (mirror ghost): a field even about the wall plane z = -1/2 has
    # zero normal gradient there, and the interior is untouched
    o3, _ = _lattice3(16, wall=1)
    x3, y3, z3 = _coords(16)
    b = np.cos(math.pi * (z3 + 0.5) / 16.0) + 0.1 * np.sin(2 * math.pi * x3 / 16)
    gb = o3.grad_field(b).reshape(3, 16, 16, 16)
    exact = -math.pi / 16 * np.sin(math.pi * (z3 + 0.5) / 16.0).reshape(16, 16, 16)
    assert np.abs(gb[2, 1:-1] - exact[1:-1]).max() < 0.01 * math.pi / 16
    assert np.abs(gb[2, 0] - exact[0]).max() < 0.02 * math.pi / 16


def test_bulk_pressure_obeys_gibbs_duhem():
    o, p = _lattice3(4)
    p.kappa1, p.kappa2, p.kappa3 = 0.011, 0.023, 0.017
    o, _ = _lattice3(4)
    o.p.kappa1, o.p.kappa2, o.p.kappa3 = 0.01, 0.02, 0.015  # (_lattice3 values; kept for clarity)
    rng = np.random.default_rng(1)
    N = o.N
    for _ in range(6):
        v = np.array([1 + 0.1 * rng.standard_normal(), rng.uniform(-1, 1), rng.uniform(0, 1)])

        def mu(vv):
            f = [np.full(N, vv[q]) for q in range(3)]
            return np.array([m[0] for m in o.potentials(f[0], f[1], f[2], f[2])])

        def pb(vv):
            return o.bulk_pressure(*vv) - CS2 * vv[0]

        h = 1e-5
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            dp = (pb(v + e) - pb(v - e)) / (2 * h)
            dmu = (mu(v + e) - mu(v - e)) / (2 * h)
            assert abs(dp - np.dot(v, dmu)) < 1e-8, (a, dp, np.dot(v, dmu))


def _smooth_state(n):
    x, y, z = _coords(n)
    k = 2 * math.pi / n
    rho = 1 + 0.03 * np.sin(k * x + 0.4) * np.cos(k * z)
    phi = 0.7 * np.sin(k * y + 0.1) * np.cos(k * (x - z))
    psi = 0.45 + 0.35 * np.cos(k * (x + 2 * y) + 0.7) * np.sin(k * z + 0.2)
    I = psi + 0.1 * np.sin(k * (y - z))
    return rho, phi, psi, I


@pytest.mark.parametrize("kappa_c", [0.0, 0.01])
def test_pressure_tensor_form_equals_potential_form(kappa_c):
    diffs = []
    for n in (48, 96):
        wl = W.small_3d(nx=n, ny=n, nz=n, wall=0)
        wl.membranes = []
        p = wl.params
        p.alpha = 1.0
        p.kappa1, p.kappa2, p.kappa3, p.kappa_c = 0.01, 0.02, 0.015, kappa_c
        Fs = []
        for form in ("potential", "pressure_tensor"):
            p.force_form = form
            o = oracle.Oracle(wl, init=False)
            Fs.append(o.force_fe(*_smooth_state(n)))
        diffs.append(np.sqrt(((Fs[1] - Fs[0]) ** 2).sum() / (Fs[0] ** 2).sum()))
    # second order (the fields resolved on twice the nodes: a quarter)
    assert diffs[1] < diffs[0] / 3.5, diffs
    assert diffs[1] < 0.012, diffs


def test_step_uses_the_selected_force_form():
    """The force of a step (read back after it) is force_fe of the state the
    step started from, in either form; the two forms' steps conserve mass."""
    for form in ("potential", "pressure_tensor"):
        wl = W.small_3d(nx=12, ny=11, nz=10, wall=0)
        wl.membranes = []
        wl.params.force_form = form
        o = oracle.Oracle(wl, init=False)
        C0, u0 = W.random_fields(wl.params, seed=2)
        o.init(C0, u0)
        fields = [o.field(n) for n in ("rho", "phi", "psi")]
        I = np.full(o.N, 0.5 * (1 + math.tanh(-wl.params.dc / (2 * wl.params.alpha))))
        Fexp = o.force_fe(*fields, I)
        m0 = o.masses()
        o.step(1)
        F = np.stack([o.field("Fx"), o.field("Fy"), o.field("Fz")])
        assert np.abs(F - Fexp).max() < 1e-15, form
        assert np.abs(o.masses() - m0).max() < 1e-12 * o.N
