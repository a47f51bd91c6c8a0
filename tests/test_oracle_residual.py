"""Pins of the oracle's equilibrium residual (the largest change of phi, psi
and of the marker positions between two checks, over the steps between
them).  The paper gives no convergence criterion (Sec. 4); the pins fix what
the definition must give on states whose evolution is known in closed form:
an exactly stationary state, a C1 slab carried by a uniform flow and a
capsule advected by it."""
import numpy as np
import pytest

import oracle as O
from paper_1906_03065_gb300 import workloads as W

U, K, ALPHA = 0.05, 10, 1.0


def _params(nx, ny):
    return W.Params(dim=2, nx=nx, ny=ny, nz=1, storage="f64", gamma_phi=0.2, gamma_psi=0.2, alpha=ALPHA,
                    kappa1=0.01, kappa2=0.01, kappa3=0.01, kappa_c=0.01, dc=8.0, interface_pos=-1.0,
                    u0=(U, 0.0, 0.0))


def test_residual_of_a_stationary_state_is_zero():
    """Uniform composition at rest is a fixed point of the scheme: every
    change, hence the residual, vanishes to round-off."""
    nx, ny = 16, 8
    wl = W.Workload("uniform", _params(nx, ny), [])
    n = nx * ny
    Cf = np.stack([np.full(n, 0.6), np.full(n, 0.4), np.zeros(n)])
    o = O.Oracle(wl, Cf=Cf, u=np.zeros((3, n)))
    o.step(K)
    r = o.residual()
    assert np.all(r <= 1e-14), r


def test_residual_of_a_translating_slab_matches_the_shifted_tanh():
    """A C1 slab between two tanh interfaces (Sec. 2.4 profile) in a uniform
    flow U moves by U*K in K steps; the largest change of phi = C1 - C2 of a
    tanh(x/(2 alpha)) profile shifted by s is 2 tanh(s/(4 alpha)), so the
    residual is that over K.  The discrete profile is a little wider than the
    continuum one, hence the 15% band; a residual that is not divided by K,
    not a maximum, or not taken against the previous check is off by far
    more."""
    nx, ny = 64, 4
    wl = W.Workload("slab", _params(nx, ny), [])
    x = np.tile(np.arange(nx, dtype=float), ny)
    phi = np.tanh((x - 16.0) / (2 * ALPHA)) - np.tanh((x - 48.0) / (2 * ALPHA)) - 1.0
    Cf = np.stack([(1 + phi) / 2, (1 - phi) / 2, np.zeros_like(phi)])
    u = np.zeros((3, nx * ny))
    u[0] = U
    o = O.Oracle(wl, Cf=Cf, u=u)
    expect = 2.0 * np.tanh(U * K / (4.0 * ALPHA))
    for _ in range(3):  # consecutive checks: each against the previous one
        o.step(K)
        dphi, dpsi, dX, r = o.residual()
        assert 0.85 * expect <= dphi <= 1.02 * expect, (dphi, expect)
        assert dpsi < 1e-3 * dphi and dX == 0.0
        assert r == pytest.approx(dphi / K, rel=1e-15)


def test_residual_of_an_advected_capsule_is_the_flow_speed():
    """Markers of a capsule in a uniform flow move with it (eqs.
    Interpolation, UpdatedXl): the largest marker displacement over K steps
    is U*K, and it dominates the residual."""
    wl = W.Workload("cap", _params(48, 48), [])
    m = W.ring(40, 8.0, (24.0, 24.0))
    m.ks, m.kb = 0.05, 0.001
    wl.membranes.append(m)
    o = O.Oracle(wl)
    for _ in range(2):
        o.step(K)
        dphi, dpsi, dX, r = o.residual()
        assert dX == pytest.approx(U * K, rel=0.01)
        assert r == pytest.approx(max(dphi, dpsi, dX) / K, rel=1e-15)
