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
