"""Host-side measures of the 2D validation experiments (no GPU): the Taylor
deformation of the equivalent ellipse, the aspect ratio and the initial
fields of the Sec. 4 set-ups, against closed forms."""
import math

import numpy as np
import pytest

from paper_1906_03065_gb300 import validation as V


def _ellipse(a, b, n=4000, phase=0.3, centre=(120.0, 60.0), tilt=0.0):
    t = phase + 2 * math.pi * np.arange(n) / n
    x, y = a * np.cos(t), b * np.sin(t)
    c, s = math.cos(tilt), math.sin(tilt)
    return np.stack([centre[0] + c * x - s * y, centre[1] + s * x + c * y, np.zeros(n)], 1)


@pytest.mark.parametrize("a,b,tilt", [(20.0, 20.0, 0.0), (24.0, 16.0, 0.0), (30.0, 10.0, 0.7)])
def test_taylor_deformation_of_ellipses(a, b, tilt):
    X = _ellipse(a, b, tilt=tilt)
    A, (cx, cy), _ = V.area_moments(X)
    assert abs(A / (math.pi * a * b) - 1) < 1e-5
    assert abs(cx - 120.0) < 1e-9 and abs(cy - 60.0) < 1e-9
    assert abs(V.taylor_deformation(X) - (a - b) / (a + b)) < 1e-6


def test_lens_deformation_of_a_sampled_ellipse_field():
    ny, nx = 120, 240
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    a, b = 30.0, 15.0
    inside = ((x - 120) / a) ** 2 + ((y - 60) / b) ** 2 <= 1
    assert abs(V.lens_deformation(inside.astype(float).ravel(), (ny, nx)) - (a - b) / (a + b)) < 5e-3


def test_aspect_ratio_and_tensions():
    X = _ellipse(24.0, 16.0)
    assert abs(V.aspect_ratio(X) - 1.5) < 1e-6
    g12, g13, g23 = V.tensions((8e-3, 8e-3, 5e-4))
    assert abs(g12 / g13 - 1.882) < 1e-3  # printed in Sec. 4.1 for the symmetric case


def test_initial_fields_sum_to_one_and_carry_the_interfaces():
    wl = V.capsule_at_interface((8e-3, 8e-3, 1e-2), 1e-3, 1e-2)
    C = V.initial_fields(wl)
    assert np.abs(C.sum(0) - 1).max() < 1e-12
    C1 = C[0].reshape(wl.params.ny, wl.params.nx)
    # C1 above mid-height, C2 below, both interfaces (60 and 0 = 120) at one half
    col = C1[:, 5]
    assert col[90] > 0.99 and col[30] < 0.01
    assert abs(col[60] - 0.5) < 0.13 and abs(0.5 * (col[0] + col[119]) - 0.5) < 0.13
    wlb, rect = V.capillary_bridge(3e-3, 1e-2)
    Cb = V.initial_fields(wlb, bridge=rect)
    assert np.abs(Cb.sum(0) - 1).max() < 1e-12
    C2 = Cb[1].reshape(wlb.params.ny, wlb.params.nx)
    assert C2[60, 120] > 0.95 and C2[5, 5] < 0.01  # (a bridge 2S = 20 wide: tanh edges 10 cells off)


class _Inst:
    def __init__(self, X):
        self.X = X

    def nodes(self, m):
        return self.X


class _StubBatch(list):
    """Stands in for a relaxed batch: instance i holds the markers the stub
    relaxation gave it."""


def _stub_relax(shape_of):
    def relax(wls, steps, fields=None, device=None):
        return _StubBatch(_Inst(shape_of(wl, steps)) for wl in wls)
    return relax


def test_deformation_sweep_rows_follow_the_batch_order(monkeypatch):
    """Every (ks, kb, kappa) capsule is one instance of a single batch; row i
    reports instance i's deformation under its own (kappa, ks, kb)."""
    cases = [(8e-3, 8e-3, 5e-4), (8e-3, 8e-3, 1e-3), (8e-3, 8e-3, 2e-3)]

    def shape(wl, steps):  # an ellipse whose D encodes the instance's ks and kappa_3
        m = wl.membranes[0]
        d = 0.1 * math.log10(1.0 / m.ks) + 10 * wl.params.kappa3
        return _ellipse(20 * (1 + d), 20 * (1 - d))

    monkeypatch.setattr(V, "relax", _stub_relax(shape))
    rows = V.deformation_sweep(cases, ks_list=(1e-3, 1e-1), kb_list=(1e-4, 1e-2), steps=10, lens=False)
    assert [(r["ks"], r["kb"], r["kappa"]) for r in rows] == \
        [(ks, kb, k) for ks in (1e-3, 1e-1) for kb in (1e-4, 1e-2) for k in cases]
    for r in rows:
        want = 0.1 * math.log10(1.0 / r["ks"]) + 10 * r["kappa"][2]
        assert abs(r["D"] - want) < 1e-6
        g12, g13, _ = V.tensions(r["kappa"])
        assert r["g12/g13"] == pytest.approx(g12 / g13)


def test_galilean_rows_measure_drift_and_shape(monkeypatch):
    """The Galilean rows take the mean marker displacement from the
    stationary run as the drift and compare the shapes with each centroid
    removed: a run translated by U * steps and uniformly offset by 0.01 in
    x has drift U * steps + 0.01 and shape deviation 0."""
    def shape(wl, steps):
        U = wl.params.u0[0]
        X = _ellipse(22.0, 18.0)
        X[:, 0] += U * steps + (0.01 if U else 0.0)
        return X

    monkeypatch.setattr(V, "relax", _stub_relax(shape))
    rows = V.galilean_runs(U_list=(1e-4, 1e-2), steps=1000)
    assert [r["U"] for r in rows] == [1e-4, 1e-2]
    for r in rows:
        assert r["drift"][0] == pytest.approx(r["U"] * 1000 + 0.01)
        assert abs(r["drift"][1]) < 1e-12
        assert r["shape_dev"] < 1e-9
        assert r["D"] == pytest.approx(r["D_stationary"])
        assert r["U_steps"] == pytest.approx(r["U"] * 1000)
