"""Equilibrium-quality measures on the GPU against the oracle (through the
C ABI): capsule area and volume of tlb_diagnostics, and the contact angle of
tlb_contact_angle.

* Read-out parity: the oracle's measures of the GPU's own state (fields and
  markers read back) equal the GPU's read-out to FP64 rounding.
* End-to-end parity: after a run, the GPU's measures equal the oracle's
  measures of the oracle's run, within what the state tolerances imply.
* A capsule centred a distance h above a flat interface meets it at
  arccos(-h/R) (closed form).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1906_03065_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_03065_gb300 import build
    build.build()
    oracle.build()


def _sim(wl):
    from paper_1906_03065_gb300 import Simulation
    return Simulation(wl)


@pytest.mark.parametrize("which", ["2d_f64", "3d_f32"])
def test_readout_matches_oracle_measures_of_the_same_state(which):
    wl = W.capsule_2d("f64") if which == "2d_f64" else W.small_3d("f32")
    g = _sim(wl).init()
    g.step(150)
    o = oracle.Oracle(wl, init=False)
    X = g.nodes(0)
    d = g.diagnostics()
    A, V = o.capsule_measures(0, X)
    assert abs(d.area[0] - A) <= 1e-12 * abs(A)
    assert abs(d.volume[0] - V) <= 1e-12 * max(abs(V), 1.0)
    ca = g.contact_angle()[0]
    (mean, lo, hi), cnt = o.contact_angle(0, X, g.field("phi"))
    assert int(ca[3]) == cnt and cnt > 0
    assert abs(ca[0] - mean) < 1e-9 and abs(ca[1] - lo) < 1e-9 and abs(ca[2] - hi) < 1e-9


def test_measures_after_a_run_match_the_oracle_run():
    wl = W.capsule_2d("f64")
    g, o = _sim(wl).init(), oracle.Oracle(wl)
    g.step(500)
    o.step(500)
    d = g.diagnostics()
    A, _ = o.capsule_measures(0)
    assert abs(d.area[0] - A) < 1e-9 * A
    (mean, _, _), cnt = o.contact_angle(0)
    ca = g.contact_angle()[0]
    assert int(ca[3]) == cnt and abs(ca[0] - mean) < 1e-8
    wl3 = W.small_3d("f32")
    g3, o3 = _sim(wl3).init(), oracle.Oracle(wl3)
    g3.step(200)
    o3.step(200)
    d3 = g3.diagnostics()
    A3, V3 = o3.capsule_measures(0)
    # markers agree to 1e-4 lattice units: area and volume to ~1e-4 * 2/R
    assert abs(d3.area[0] / A3 - 1) < 1e-4 and abs(d3.volume[0] / V3 - 1) < 1e-4
    (m3, _, _), c3 = o3.contact_angle(0)
    ca3 = g3.contact_angle()[0]
    assert int(ca3[3]) == c3 and abs(ca3[0] - m3) < 0.05


@pytest.mark.parametrize("h", [0.37, 3.0])
def test_contact_angle_closed_form(h):
    """Fluid started as a flat tanh interface phi = tanh((z - z0)/(2 alpha))
    (C1 above, C2 below, no C3): a sphere centred at z0 + h meets it at
    arccos(-h/R); the oracle's read-out of the same state agrees to FP64
    rounding of the FP32 fields.  (h = 0 would put icosphere vertices on the
    plane itself, where phi = 0 up to rounding and whether an edge holds a
    contact point is decided by the last bit.)"""
    n, R = 64, 20.0
    wl = W.capsule_3d("f32", n=n, level=4, radius=R)
    wl.membranes[0].X = wl.membranes[0].X + np.array([0.31, -0.17, h])
    z = np.repeat(np.arange(n), n * n).astype(float)
    s = 0.5 * (1 + np.tanh((z - n / 2) / (2 * wl.params.alpha)))
    C = np.stack([s, 1 - s, np.zeros_like(s)])
    g = _sim(wl)
    g.init(C, None)
    mean, lo, hi, cnt = g.contact_angle()[0]
    assert cnt > 30
    assert abs(mean - math.degrees(math.acos(-h / R))) < 0.1, mean
    o = oracle.Oracle(wl, init=False)
    (om, _, _), oc = o.contact_angle(0, g.nodes(0), g.field("phi"))
    assert oc == int(cnt) and abs(om - mean) < 1e-9
    # area and volume of the initial icosphere: the oracle's closed-form-pinned measures
    A, V = o.capsule_measures(0, wl.membranes[0].X)
    d = g.diagnostics()
    assert abs(d.area[0] - A) < 1e-12 * A and abs(d.volume[0] - V) < 1e-12 * V
