"""Learned warm start on the GPU: the library's forward pass, gradients and
Adam step against the FP64 reference network of oracle/warmstart.py (which
rounds stored activations to bf16 as the GPU stores them), the warm start of
a context (mass-projected fields, moved markers), and a small end-to-end
run: relax a few instances, train on them, relax held-out instances from the
plain and from the learned start."""
import numpy as np
import pytest

from oracle import warmstart as ws
from paper_1906_03065_gb300 import workloads as W

pytestmark = pytest.mark.gpu

E, C0, LV = 16, 16, 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_03065_gb300 import build
    build.build()
    import oracle
    oracle.build()


def _theta(seed, c0=C0, lv=LV):
    rng = np.random.default_rng(seed)
    th = ws.init_params(seed, c0, lv)
    o = 0
    for t, ci, co in ws.layer_shapes(c0, lv):
        o += t * ci * co
        th[o:o + co] = rng.normal(0, 0.05, co)  # live biases
        o += co
    th[o - 16 - c0 * 16:o - 16] = rng.normal(0, 0.2, c0 * 16)  # live output layer
    return th


def _inputs(rng, B, e=E):
    xs = [ws.make_input(rng.uniform(-1, 1, e ** 3), rng.uniform(0, 1, e ** 3), rng.uniform(-1, 1, 5), e)
          for _ in range(B)]
    return np.stack(xs)


def _to_gpu_x(x):
    import torch
    B, Cn = x.shape[0], x.shape[1]
    xl = np.ascontiguousarray(x.reshape(B, Cn, -1).transpose(0, 2, 1))
    return torch.from_numpy(xl).to(torch.bfloat16).cuda()


def _net(**kw):
    from paper_1906_03065_gb300 import WarmStartNet
    d = dict(edge=E, base_channels=C0, levels=LV, max_batch=4, max_nodes=32)
    d.update(kw)
    return WarmStartNet(**d)


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_forward_matches_oracle():
    rng = np.random.default_rng(0)
    th = _theta(1)
    x = _inputs(rng, 2)
    net = _net()
    net.set_params(th)
    y = net.forward(_to_gpu_x(x)).cpu().numpy()
    yo, _ = ws.forward(th, x, c0=C0, levels=LV)
    yo = yo.numpy().reshape(2, 16, -1).transpose(0, 2, 1)
    assert _relerr(y[..., :5], yo[..., :5]) < 5e-3
    assert np.abs(y - yo).max() < 2e-2 * np.abs(yo).max()
    assert net.launches() > 0


@pytest.mark.parametrize("c0,lv,e", [(16, 3, 16), (48, 2, 24)])
def test_tcgen05_convolutions_match_the_mma_sync_path(c0, lv, e):
    """The 3x3x3 convolutions on tcgen05 (tensor-memory accumulators; operands
    staged by cp.async or loaded by TMA) against the mma.sync path on the same
    bf16 operands: the two differ only in the
    order of the FP32 accumulation (and the bf16 roundings that follows).
    Channel counts 16..192 take every column tile (16, 32, 64); edges 24, 12,
    16, 8, 4 leave ragged bricks."""
    import torch
    rng = np.random.default_rng(5)
    th = _theta(7, c0, lv)
    x = _to_gpu_x(_inputs(rng, 2, e))
    B, n = 2, 10
    dphi = torch.from_numpy(rng.normal(0, 0.05, (B, e ** 3)).astype(np.float32)).cuda()
    dpsi = torch.from_numpy(rng.normal(0, 0.05, (B, e ** 3)).astype(np.float32)).cuda()
    out = []
    for mode in (0, 1, 2):  # mma.sync, tcgen05 with cp.async staging, tcgen05 fed by TMA
        net = _net(edge=e, base_channels=c0, levels=lv, max_batch=2, max_nodes=0)
        net.set_tcgen05(mode)
        net.set_params(th)
        y = net.forward(x).cpu().numpy()
        L = net.train_step(x, dphi, dpsi, None, None, None, lam=0.0, lr=1e-3, update=False)
        assert net.status() == 0
        out.append((y, L, net.grads()))
    ya, La, ga = out[0]
    for yb, Lb, gb in out[1:]:
        assert _relerr(yb, ya) < 3e-3
        assert Lb == pytest.approx(La, rel=1e-3)
        assert _relerr(gb, ga) < 1e-2
    # the two tcgen05 paths issue the same products in the same order
    assert np.array_equal(out[1][0], out[2][0])


def test_gradients_and_adam_match_oracle():
    import torch
    rng = np.random.default_rng(2)
    th = _theta(3)
    B, n = 2, 20
    x = _inputs(rng, B)
    dphi = rng.normal(0, 0.05, (B, E ** 3))
    dpsi = rng.normal(0, 0.05, (B, E ** 3))
    X0 = [rng.uniform(1, E - 2, (n, 3)) for _ in range(B)]
    off = [rng.normal(0, 0.2, (n, 3)) for _ in range(B)]
    net = _net()
    net.set_params(th)
    Xa = np.zeros((B, 32, 3), np.float32)
    Oa = np.zeros((B, 32, 3), np.float32)
    for b in range(B):
        Xa[b, :n], Oa[b, :n] = X0[b], off[b]
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    L = net.train_step(_to_gpu_x(x), f(dphi), f(dpsi), f(Xa), f(Oa), [n] * B, lam=0.5, lr=1e-3, update=False)
    Lo = ws.loss(th, x, dphi, dpsi, X0, off, lam=0.5, c0=C0, levels=LV).item()
    assert L == pytest.approx(Lo, rel=1e-2)
    g = net.grads()
    go = ws.grad(th, x, dphi, dpsi, X0, off, lam=0.5, c0=C0, levels=LV)
    # per weight and bias tensor (bf16 GEMM operands against FP64 backward);
    # tensors whose gradient is negligible beside the largest are skipped
    o, big = 0, np.abs(go).max()
    for k, (t, ci, co) in enumerate(ws.layer_shapes(C0, LV)):
        nw = t * ci * co
        for s in (slice(o, o + nw), slice(o + nw, o + nw + co)):
            if np.abs(go[s]).max() > 1e-3 * big:
                assert _relerr(g[s], go[s]) < 4e-2, (k, s, _relerr(g[s], go[s]))
        o += nw + co
    assert _relerr(g, go) < 2e-2
    # one Adam step (update=1) from the same state
    net.set_params(th)
    net.train_step(_to_gpu_x(x), f(dphi), f(dpsi), f(Xa), f(Oa), [n] * B, lam=0.5, lr=1e-3, update=True)
    g1 = net.grads()
    t1 = net.params()
    ref, _, _ = ws.adam(th.astype(np.float64), g1.astype(np.float64), np.zeros_like(g1, dtype=np.float64),
                        np.zeros_like(g1, dtype=np.float64), 1, lr=1e-3)
    assert np.abs(t1 - ref).max() < 1e-6


def test_training_steps_are_bitwise_reproducible():
    """The marker loss scatters its gradient in fixed point, so the same
    training steps from the same state give the same parameters bit for bit,
    even with many markers sharing voxels."""
    import torch
    rng = np.random.default_rng(4)
    B, n = 2, 32
    x = _to_gpu_x(_inputs(rng, B))
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    dphi, dpsi = f(rng.normal(0, 0.05, (B, E ** 3))), f(rng.normal(0, 0.05, (B, E ** 3)))
    X0 = f(rng.uniform(7.0, 8.5, (B, n, 3)))  # every marker in the same few voxels
    off = f(rng.normal(0, 0.2, (B, n, 3)))
    out = []
    for _ in range(2):
        net = _net()
        net.set_params(_theta(5))
        for _ in range(3):
            net.train_step(x, dphi, dpsi, X0, off, [n] * B, lam=1.0, lr=1e-3, update=True)
        out.append((net.params(), net.grads()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def _cube(edge=32, R=6.0, level=2, seed=0):
    rng = np.random.default_rng(seed)
    c = edge / 2.0
    k = rng.uniform(0.005, 0.03, 3)
    p = W.Params(dim=3, nx=edge, ny=edge, nz=edge, wall_last=1, storage="f32", alpha=1.0, kappa1=k[0],
                 kappa2=k[1], kappa3=k[2], kappa_c=0.01, dc=8.0, interface_pos=c)
    m = W.icosphere(level, R * rng.uniform(0.9, 1.1), (c + rng.uniform(-0.4, 0.4), c + rng.uniform(-0.4, 0.4), c))
    m.G, m.C, m.kb = float(rng.uniform(0.002, 0.05)), 1.0, 0.005
    return W.Workload(f"cube{edge}_{seed}", p, [m], steps=0)


def test_warm_start_of_a_context():
    """Markers move by the mean predicted displacement plus its normal part;
    psi becomes the profile of the moved markers and phi = (1 - psi)(s0 + y0),
    both shifted to the plain totals; the context then holds the equilibrium
    populations of these fields (compared with the FP64 reference of the
    same composition, oracle.warmstart)."""
    import oracle
    from paper_1906_03065_gb300 import Simulation, warmstart as WS
    wl = _cube(32)
    th = _theta(5, lv=3)
    net = _net(edge=32, max_batch=1)
    net.set_params(th)
    s = Simulation(wl).init()
    phi0, psi0, X0 = s.field("phi"), s.field("psi"), s.nodes(0)
    feats = WS.features(wl)
    net.warm_start(s, feats)
    o = oracle.Oracle(wl)
    x = ws.make_input(o.field("phi"), o.field("psi"), feats, 32)[None]
    yo, _ = ws.forward(th, x, c0=C0, levels=3)
    yo = yo[0].numpy()
    F = wl.membranes[0].elems
    Xr = ws.warm_start_markers(yo, X0, ws.vertex_normals(X0, F), F)
    # the moved membrane encloses the plain start's volume
    assert abs(ws.enclosed_volume(s.nodes(0), F) / ws.enclosed_volume(X0, F) - 1) < 1e-9
    D = np.abs(Xr - X0).max()
    assert D > 0.05  # the test moves the markers
    assert np.abs(s.nodes(0) - Xr).max() < 5e-3 * D + 1e-5
    I_new, _, _ = o.iprofile(Xr)
    p_ref, s_ref, l_psi, l_phi = ws.warm_start_fields(yo[0].reshape(-1), phi0, psi0, I_new, factors=True)
    # the bf16 forward pass agrees with the FP64 reference to 2% of max |y|
    # (test_forward_matches_oracle); phi = (1 - psi)(s + l_phi (1 - s^2)_+)
    # carries an error e of s as (1 + 2 |l_phi| |s|) e, and psi = I (1 + l_psi
    # 4 (1 - I)) an error of I as (1 + 4 |l_psi|)
    tol = 2e-3 + 2e-2 * np.abs(yo[0]).max()
    smax = np.abs(yo[0]).max() + 1.0
    assert np.abs(s.field("psi") - s_ref).max() < tol * (1 + 4 * abs(l_psi))
    assert np.abs(s.field("phi") - p_ref).max() < tol * (1 + 2 * abs(l_phi) * smax) * (1 + 4 * abs(l_psi))
    assert s.field("phi").sum() == pytest.approx(phi0.sum(), abs=1e-2)
    assert s.field("psi").sum() == pytest.approx(psi0.sum(), abs=1e-2)
    s.step(5)  # the relaxation runs from it
    assert np.isfinite(s.field("C3")).all()


def test_training_gains_over_the_plain_start():
    """Relax 12 instances, train on 10, then relax the 2 held-out instances
    from the plain and from the learned start: the learned start is closer
    to equilibrium (smaller residual over the first checks)."""
    from paper_1906_03065_gb300 import WarmStartNet, warmstart as WS
    wls = [_cube(32, seed=100 + i) for i in range(12)]
    net = WarmStartNet(edge=32, base_channels=16, levels=3, max_batch=4, max_nodes=162)
    net.set_params(ws.init_params(0, 16, 3))
    data = WS.dataset(net, wls[:10], max_steps=1500, check_every=500, tol=0.0)
    losses = WS.train(net, data, epochs=40, batch=4, lr=2e-3)
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:3])
    r = WS.compare(net, wls[10:], max_steps=300, check_every=300, tols=(1e-12,))
    plain, learned = r["plain"]["history"][0], r["learned"]["history"][0]
    assert np.mean(learned) < np.mean(plain), (plain, learned)
