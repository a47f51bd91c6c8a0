"""Pins of the oracle's membrane energies and forces (no GPU).

* forces equal minus the central finite-difference gradient of the energies
  (eq. MembraneForces: F = -dE/dX),
* closed forms: regular polygon stretching and bending (eqs. DiscreteSE,
  DiscreteBE, DiscreteTheta), uniform dilation of a Skalak membrane, the
  Helfrich energy of a sphere (8 pi kb),
* internal forces carry no net force and no net torque.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1906_03065_gb300 import workloads as W


def _fd_grad(E, X, idx, h=1e-6):
    out = []
    for (l, k) in idx:
        Xp = X.copy(); Xp[l, k] += h
        Xm = X.copy(); Xm[l, k] -= h
        out.append((E(Xp) - E(Xm)) / (2 * h))
    return np.array(out)


def _ring_oracle(n=24, radius=5.0, jitter=0.3, seed=0):
    wl = W.small_2d(nx=24, ny=24, nodes=n, radius=radius, centre=(12.0, 12.0))
    wl.membranes[0].ks, wl.membranes[0].kb = 0.07, 0.013
    o = oracle.Oracle(wl, init=False)
    X = W.jitter_nodes(wl.membranes[0], jitter, seed).X if jitter else wl.membranes[0].X.copy()
    return o, X, wl


def _sphere_oracle(level=2, radius=6.0, jitter=0.2, seed=0, G=0.013, C=0.7, kb=0.004):
    wl = W.small_3d(nx=24, ny=24, nz=24, level=level, radius=radius, centre=(12.0, 12.0, 12.0))
    m = wl.membranes[0]
    m.G, m.C, m.kb = G, C, kb
    o = oracle.Oracle(wl, init=False)
    X = W.jitter_nodes(m, jitter, seed).X if jitter else m.X.copy()
    return o, X, wl


@pytest.mark.parametrize("which", [0, 1])
def test_ring_forces_are_minus_gradient(which):
    o, X, _ = _ring_oracle()
    F = o.mem_force(0, which, X)
    idx = [(l, k) for l in (0, 3, 11, 23) for k in (0, 1)]
    g = _fd_grad(lambda Y: o.mem_energy(0, which, Y), X, idx)
    Fi = np.array([F[l, k] for (l, k) in idx])
    assert np.abs(Fi + g).max() <= 1e-7 * np.abs(F).max()


@pytest.mark.parametrize("which", [0, 1])
def test_sphere_forces_are_minus_gradient(which):
    o, X, _ = _sphere_oracle()
    F = o.mem_force(0, which, X)
    idx = [(l, k) for l in (0, 5, 40, 97, 161) for k in (0, 1, 2)]
    g = _fd_grad(lambda Y: o.mem_energy(0, which, Y), X, idx)
    Fi = np.array([F[l, k] for (l, k) in idx])
    assert np.abs(Fi + g).max() <= 1e-6 * np.abs(F).max()


@pytest.mark.parametrize("kind", ["ring", "sphere"])
def test_internal_forces_balance(kind):
    """Translation and rotation invariance of the elastic energies: zero net
    force and zero net torque."""
    o, X, _ = _ring_oracle() if kind == "ring" else _sphere_oracle()
    for which in (0, 1):
        F = o.mem_force(0, which, X)
        scale = np.abs(F).max()
        assert np.abs(F.sum(0)).max() <= 1e-12 * scale * len(X)
        c = X - X.mean(0)
        assert np.abs(np.cross(c, F).sum(0)).max() <= 1e-11 * scale * len(X) * np.abs(c).max()


def test_regular_polygon_closed_forms():
    """Regular N-gon of side a scaled from rest side a0: Es = ks/2 N (a/a0 - 1)^2 a0
    and, with Delta theta = 4 pi / N (twice the turning angle) and
    Delta s' = 2a, Eb = kb/4 N (4 pi/N)^2 / (2a) = 2 pi^2 kb / (N a)."""
    n, R = 76, 12.0
    wl = W.capsule_2d()
    m = wl.membranes[0]
    o = oracle.Oracle(wl, init=False)
    a0 = 2 * R * math.sin(math.pi / n)
    assert abs(a0 - 0.991799) < 1e-6
    for scale in (1.0, 1.05):
        X = m.X.copy()
        X[:, :2] = 32 + (X[:, :2] - 32) * scale
        a = a0 * scale
        Es = o.mem_energy(0, 0, X)
        Eb = o.mem_energy(0, 1, X)
        assert abs(Es - m.ks / 2 * n * (a / a0 - 1) ** 2 * a0) <= 1e-12 + 1e-9 * Es
        assert abs(Eb - 2 * math.pi ** 2 * m.kb / (n * a)) <= 1e-12 * 1e3
    # the value quoted for the 76-marker ring at R = 12
    assert abs(o.mem_energy(0, 1, m.X) / m.kb - 0.261874) < 1e-6


def test_skalak_uniform_dilation_closed_form():
    """Uniform dilation by lambda of the reference mesh: every triangle has
    C^ = lambda^2 I, so I1 = 2 lambda^2 - 2, I2 = lambda^4 - 1 and
    E = A0 (G/4)(I1^2 + 2 I1 - 2 I2 + C I2^2); zero energy and force at rest."""
    o, X0, wl = _sphere_oracle(jitter=0.0)
    m = wl.membranes[0]
    T = m.elems
    A0 = 0.5 * np.linalg.norm(np.cross(X0[T[:, 1]] - X0[T[:, 0]], X0[T[:, 2]] - X0[T[:, 0]]), axis=1).sum()
    assert abs(o.mem_energy(0, 0, X0)) < 1e-13
    assert np.abs(o.mem_force(0, 0, X0)).max() < 1e-14
    c = X0.mean(0)
    for lam in (0.9, 1.1, 1.3):
        X = c + lam * (X0 - c)
        I1, I2 = 2 * lam ** 2 - 2, lam ** 4 - 1
        ref = A0 * m.G / 4 * (I1 ** 2 + 2 * I1 - 2 * I2 + m.C * I2 ** 2)
        assert abs(o.mem_energy(0, 0, X) - ref) <= 1e-12 * abs(ref)


def test_helfrich_sphere_energy_converges_to_8_pi_kb():
    """Helfrich energy of a sphere, (kb/2) int (2H)^2 dA = 8 pi kb, independent
    of the radius; the discrete value approaches it under refinement."""
    errs = []
    for level in (2, 3, 4):
        o, X, wl = _sphere_oracle(level=level, radius=7.0, jitter=0.0)
        E = o.mem_energy(0, 1, X)
        errs.append(abs(E / (8 * math.pi * wl.membranes[0].kb) - 1))
    assert errs[-1] < 0.01
    assert errs[0] > errs[1] > errs[2]
