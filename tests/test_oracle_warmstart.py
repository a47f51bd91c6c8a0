"""Pins of the warm-start network's CPU reference (oracle/warmstart.py):
bf16 rounding against torch's conversion, the tap convention of a conv
against a plain shift, trilinear sampling exact for linear fields, the
gradient against central finite differences, Adam's first step (size lr in
every coordinate), the mass projection, and an untrained output layer that
returns the plain start."""
import numpy as np
import pytest
import torch

from oracle import warmstart as ws

C0, LV, E = 16, 2, 8


def _sample(rng, B=2, n=6):
    x = np.stack([ws.make_input(rng.uniform(-1, 1, E ** 3), rng.uniform(0, 1, E ** 3),
                                rng.uniform(-1, 1, 5), E) for _ in range(B)])
    X0 = [rng.uniform(0.5, E - 1.5, (n, 3)) for _ in range(B)]
    return x, X0


def test_round_bf16_matches_torch():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(0, 1, 1000), rng.normal(0, 1e-30, 100), [0.0, -0.0, 1e38, -3.0e38, 1.0 + 2 ** -8,
                        1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9]])
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ws.round_bf16(v), ref)


def test_conv_tap_convention_is_a_shift():
    """A conv whose only weight is 1 at tap (kz, ky, kx), ci = co = 0 returns
    the input at the offset (kz-1, ky-1, kx-1), zero outside."""
    rng = np.random.default_rng(1)
    h = torch.from_numpy(rng.normal(0, 1, (1, 16, E, E, E)))
    for tap in (0, 5, 13, 22, 26):
        W = torch.zeros(27, 16, 16, dtype=torch.float64)
        W[tap, 0, 0] = 1.0
        out = ws._conv(h, W, torch.zeros(16, dtype=torch.float64), 27)[0, 0].numpy()
        dz, dy, dx = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
        ref = np.zeros((E, E, E))
        src = h[0, 0].numpy()
        for z in range(E):
            for y in range(E):
                for x in range(E):
                    if 0 <= z + dz < E and 0 <= y + dy < E and 0 <= x + dx < E:
                        ref[z, y, x] = src[z + dz, y + dy, x + dx]
        assert np.array_equal(out, ref), tap


def test_trilinear_is_exact_for_linear_fields():
    rng = np.random.default_rng(2)
    z, y, x = np.meshgrid(np.arange(E), np.arange(E), np.arange(E), indexing="ij")
    a = rng.normal(0, 1, (3, 4))
    D = torch.from_numpy(np.stack([a[k, 0] * x + a[k, 1] * y + a[k, 2] * z + a[k, 3] for k in range(3)]))
    X = rng.uniform(0, E - 1, (50, 3))
    got = ws.trilinear(D, torch.from_numpy(X)).numpy()
    ref = np.stack([a[k, 0] * X[:, 0] + a[k, 1] * X[:, 1] + a[k, 2] * X[:, 2] + a[k, 3] for k in range(3)], axis=1)
    assert np.abs(got - ref).max() < 1e-12


def test_gradient_matches_finite_differences():
    """dL/dtheta by reverse mode against central differences of the FP64 loss
    (no bf16 rounding) for parameters of every layer kind."""
    rng = np.random.default_rng(3)
    theta = ws.init_params(4, C0, LV).astype(np.float64)
    theta[-(16 * 16 + 16):] = rng.normal(0, 0.1, 16 * 16 + 16)  # a live output layer
    x, X0 = _sample(rng)
    dphi = rng.normal(0, 0.1, (2, E ** 3))
    dpsi = rng.normal(0, 0.1, (2, E ** 3))
    off = [rng.normal(0, 0.3, (6, 3)) for _ in range(2)]
    args = (x, dphi, dpsi, X0, off)
    kw = dict(lam=0.7, bf16=False, c0=C0, levels=LV)
    g = ws.grad(theta, *args, **kw)
    offs, o = [], 0
    for t, ci, co in ws.layer_shapes(C0, LV):
        offs += [o + rng.integers(0, t * ci * co), o + t * ci * co + rng.integers(0, co)]
        o += t * ci * co + co
    h = 1e-6
    for i in offs:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (ws.loss(tp, *args, **kw).item() - ws.loss(tm, *args, **kw).item()) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_adam_first_step_has_size_lr():
    rng = np.random.default_rng(5)
    th = rng.normal(0, 1, 100)
    g = rng.normal(0, 1, 100)
    t1, m, v = ws.adam(th, g, np.zeros(100), np.zeros(100), 1, lr=1e-3)
    assert np.allclose(th - t1, 1e-3 * np.sign(g), rtol=1e-6)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_mass_projection_restores_totals():
    rng = np.random.default_rng(6)
    p0, s0 = rng.uniform(-1, 1, 500), rng.uniform(0, 1, 500)
    p, s = ws.mass_projection(p0 + rng.normal(0, 0.1, 500), s0 + 0.05, p0, s0)
    assert p.sum() == pytest.approx(p0.sum(), abs=1e-9) and s.sum() == pytest.approx(s0.sum(), abs=1e-9)
    d = s - (s0 + 0.05)
    assert np.allclose(d, d[0])


def test_untrained_output_layer_returns_plain_start():
    rng = np.random.default_rng(7)
    theta = ws.init_params(8, C0, LV)
    x, X0 = _sample(rng)
    y, offs = ws.forward(theta, x, X0, c0=C0, levels=LV)
    assert float(torch.abs(y).max()) == 0.0 and all(float(torch.abs(o).max()) == 0.0 for o in offs)


def test_warm_start_composition_pins():
    """The reference warm start conserves the phi and psi totals, returns the
    plain start for a zero output, and moves markers by a uniform
    displacement field exactly (translation only)."""
    from paper_1906_03065_gb300 import workloads as W
    rng = np.random.default_rng(9)
    m = W.icosphere(2, 5.0, (8.1, 7.9, 8.2))
    n = ws.vertex_normals(m.X, m.elems)
    radial = (m.X - m.X.mean(0)) / np.linalg.norm(m.X - m.X.mean(0), axis=1, keepdims=True)
    assert np.abs(n - radial).max() < 0.05  # sphere: close to radial
    y = np.zeros((16, E * 2, E * 2, E * 2))
    assert np.abs(ws.warm_start_markers(y, m.X, n) - m.X).max() == 0.0
    y[2], y[3], y[4] = 0.3, -0.2, 0.7
    assert np.abs(ws.warm_start_markers(y, m.X, n) - (m.X + [0.3, -0.2, 0.7])).max() < 1e-12
    psi0 = rng.uniform(0, 1, 300)
    phi0 = (1 - psi0) * rng.uniform(-1, 1, 300)
    phi, psi = ws.warm_start_fields(np.zeros(300), phi0, psi0, psi0)
    assert np.allclose(phi, phi0, atol=1e-12) and np.allclose(psi, psi0, atol=1e-12)
    I_new = np.clip(psi0 + rng.normal(0, 0.05, 300), 0, 1)
    phi, psi = ws.warm_start_fields(rng.normal(0, 0.1, 300), phi0, psi0, I_new)
    assert phi.sum() == pytest.approx(phi0.sum(), abs=1e-10) and psi.sum() == pytest.approx(psi0.sum(), abs=1e-10)
    # the totals are restored on the interfaces only: bulk cells (I = 0 or 1,
    # s = +-1) keep their values
    I_b = I_new.copy()
    I_b[:100], I_b[100:150] = 0.0, 1.0
    w0 = 1 - psi0
    s0 = phi0 / w0
    y0 = rng.normal(0, 0.1, 300)
    y0[150:200] = 1.0 - s0[150:200]
    y0[200:230] = -1.0 - s0[200:230]
    phi, psi = ws.warm_start_fields(y0, phi0, psi0, I_b)
    assert np.all(psi[:100] == 0.0) and np.all(psi[100:150] == 1.0)
    assert np.allclose(phi[150:200], 1 - psi[150:200], atol=1e-14)
    assert np.allclose(phi[200:230], -(1 - psi[200:230]), atol=1e-14)
    assert phi.sum() == pytest.approx(phi0.sum(), abs=1e-10) and psi.sum() == pytest.approx(psi0.sum(), abs=1e-10)


def test_enclosed_volume_and_the_volume_projection():
    """The reference warm start projects the moved markers back to the plain
    start's enclosed volume: the divergence-theorem volume of the regular
    icosahedron has its closed form, and the projection restores it."""
    import math
    from paper_1906_03065_gb300 import workloads as Wk
    R = 5.0
    m = Wk.icosphere(0, R, (12.0, 11.0, 10.0))
    a = 4 * R / math.sqrt(10 + 2 * math.sqrt(5))
    assert abs(ws.enclosed_volume(m.X, m.elems) - 5 / 12 * (3 + math.sqrt(5)) * a ** 3) < 1e-10
    m3 = Wk.icosphere(2, R, (16.0, 16.0, 16.0))
    E = 32
    y = np.zeros((16, E, E, E))
    y[2:5] = np.random.default_rng(0).normal(0.0, 0.3, (3, E, E, E))  # a non-uniform displacement field
    nrm = ws.vertex_normals(m3.X, m3.elems)
    X1 = ws.warm_start_markers(y, m3.X, nrm)
    X2 = ws.warm_start_markers(y, m3.X, nrm, m3.elems)
    V0 = ws.enclosed_volume(m3.X, m3.elems)
    assert abs(ws.enclosed_volume(X1, m3.elems) / V0 - 1) > 1e-4  # the displacement changes it
    assert abs(ws.enclosed_volume(X2, m3.elems) / V0 - 1) < 1e-12
