"""Learned warm start: training pairs from the batched relaxation, training
with the library's own kernels, and the relaxation time from the plain and
from the learned start.

The network, its forward and backward kernels, the optimiser and the warm
start itself are in the library (``tlb_net_*`` in include/tlb.h); this
module only orchestrates calls and moves tensors.  A training pair is the
plain initial state of an instance (undeformed capsule on the flat
interface) and the state the lattice Boltzmann + immersed boundary
relaxation reaches from it.
"""
from __future__ import annotations

import numpy as np

from . import Batch, WarmStartNet, workloads as W


def features(wl) -> np.ndarray:
    """The network's five inputs besides the fields: kappa_1..3, Skalak G and
    R / E, each mapped to about [-1, 1] over the sweep ranges (kappa in
    [0.005, 0.03], G in [0.002, 0.05], R / E in [0.15, 0.25])."""
    p, m = wl.params, wl.membranes[0]
    R = float(np.linalg.norm(m.X - m.X.mean(axis=0), axis=1).mean())
    return np.array([(p.kappa1 - 0.0175) / 0.0125, (p.kappa2 - 0.0175) / 0.0125, (p.kappa3 - 0.0175) / 0.0125,
                     (m.G - 0.026) / 0.024, (R / p.nx - 0.2) / 0.05])


def indicator(phi, psi):
    """Phase indicator of the C1/C2 fluid, s = phi / (1 - psi) (C1 - C2 over
    C1 + C2 when rho = 1); 0 where 1 - psi < 1e-6."""
    w = 1.0 - psi
    return np.where(w > 1e-6, phi / np.where(w > 1e-6, w, 1.0), 0.0)


def indicator_target(phi0, psi0, phi, psi, cut: float = 0.05):
    """Training target of output y0: s(equilibrium) - s(plain start), where
    the equilibrium has at least ``cut`` of non-C3 fluid (0 inside the
    capsule, where s is undefined), clipped to [-1.5, 1.5]."""
    s0 = indicator(phi0, psi0)
    s = np.clip(indicator(phi, psi), -1.5, 1.5)
    return np.where(1.0 - psi >= cut, s - s0, 0.0).astype(np.float32)


def init_params(net: WarmStartNet, seed: int) -> np.ndarray:
    """He-normal weights (standard deviation sqrt(2 / fan_in), fan_in = taps
    * input channels) from numpy's PCG64 with ``seed``, zero biases and a zero
    output layer, so that the untrained network returns the plain start.
    Layer shapes follow the network of tlb.h."""
    d = net.desc
    c = [d.base_channels << l for l in range(d.levels)]
    shapes = [(27, 16, c[0]), (27, c[0], c[0])]
    for l in range(1, d.levels):
        shapes += [(27, c[l - 1], c[l]), (27, c[l], c[l])]
    for l in range(d.levels - 2, -1, -1):
        shapes += [(27, c[l + 1] + c[l], c[l]), (27, c[l], c[l])]
    shapes.append((1, c[0], 16))
    rng = np.random.default_rng(seed)
    out = []
    for k, (t, ci, co) in enumerate(shapes):
        w = np.zeros(t * ci * co) if k == len(shapes) - 1 else rng.normal(0.0, np.sqrt(2.0 / (t * ci)), t * ci * co)
        out += [w, np.zeros(co)]
    theta = np.concatenate(out).astype(np.float32)
    assert theta.size == net.n_params
    return theta


def instances(n: int, seed: int, edge: int = 48, storage: str = "f32"):
    """``n`` sweep instances of one lattice edge (workloads.sweep_3d with a
    single edge, so every sample has the network's lattice)."""
    return W.sweep_3d(n, seed=seed, storage=storage, edges=(edge,))


def dataset(net: WarmStartNet, wls, max_steps: int, check_every: int = 200, tol: float = 1e-7):
    """Training tensors (on the net's device) of the instances ``wls``: the
    inputs of their plain starts and the targets of the outputs after relaxing
    them together as a batch to the residual ``tol`` (or ``max_steps``): the
    change of the phase indicator (``indicator_target``) for y0, zero for y1,
    and the marker offsets.  Returns a dict with x, dphi (y0 targets), dpsi
    (y1 targets), X0, off, n_nodes, steps, residual."""
    import torch
    n, V = len(wls), net.edge ** 3
    b = Batch(wls, device=net.device).init()
    dev = net.device
    x = torch.empty((n, V, 16), dtype=torch.bfloat16, device=dev)
    phi0, psi0, X0 = [], [], []
    for i, wl in enumerate(wls):
        s = b[i]
        net.input(s, features(wl), out=x[i])
        phi0.append(s.field("phi"))
        psi0.append(s.field("psi"))
        X0.append(s.nodes(0))
    steps, res = b.run(max_steps, check_every, tol)
    mn = max(net.max_nodes, 1)
    dphi = np.zeros((n, V), dtype=np.float32)
    dpsi = np.zeros((n, V), dtype=np.float32)
    Xa = np.zeros((n, mn, 3), dtype=np.float32)
    off = np.zeros((n, mn, 3), dtype=np.float32)
    nn = []
    for i in range(n):
        s = b[i]
        dphi[i] = indicator_target(phi0[i], psi0[i], s.field("phi"), s.field("psi"))
        dpsi[i] = 0.0  # psi is not predicted: the warm start takes the profile of the moved markers
        Xe = s.nodes(0)
        k = min(len(Xe), mn)
        Xa[i, :k] = X0[i][:k]
        off[i, :k] = (Xe - X0[i])[:k]
        nn.append(k if net.max_nodes else 0)
    del b
    torch.cuda.empty_cache()
    t = lambda a: torch.from_numpy(a).to(dev)  # noqa: E731
    return {"x": x, "dphi": t(dphi), "dpsi": t(dpsi), "X0": t(Xa), "off": t(off), "n_nodes": np.array(nn),
            "steps": steps, "residual": res}


def train(net: WarmStartNet, data, epochs: int, batch: int = 4, lr: float = 1e-3, lam: float = 1.0,
          seed: int = 0, lr_final: float = None):
    """Adam on random minibatches; the step size decays geometrically from
    lr to lr_final (default lr / 10).  Returns the loss of every step."""
    import torch
    rng = np.random.default_rng(seed)
    n = data["x"].shape[0]
    batch = min(batch, net.max_batch, n)
    nsteps = epochs * max(1, n // batch)
    lr_final = lr / 10 if lr_final is None else lr_final
    losses = []
    k = 0
    for _ in range(epochs):
        perm = rng.permutation(n)
        for j in range(0, n - batch + 1, batch):
            idx = torch.as_tensor(perm[j:j + batch], device=net.device)
            step_lr = lr * (lr_final / lr) ** (k / max(1, nsteps - 1))
            L = net.train_step(data["x"][idx].contiguous(), data["dphi"][idx].contiguous(),
                               data["dpsi"][idx].contiguous(), data["X0"][idx].contiguous(),
                               data["off"][idx].contiguous(), data["n_nodes"][perm[j:j + batch]],
                               lam=lam, lr=step_lr)
            losses.append(L)
            k += 1
    return losses


def measures(s) -> np.ndarray:
    """Equilibrium-quality measures of one instance: the mean contact angle
    of the capsule with the C1/C2 interface (degrees, FP64 read-out of the
    library) and the capsule's area and volume (FP64 diagnostics)."""
    d = s.diagnostics()
    return np.array([s.contact_angle()[0][0], d.area[0], d.volume[0]])


def histories(b, max_steps: int, check_every: int, stop_tol: float):
    """Residual and measures of every instance of batch ``b`` after each
    chunk of ``check_every`` steps (no instance retires) until every
    instance has reached ``stop_tol`` once or ``max_steps`` steps.  Returns
    the residuals [checks][n] and the measures [checks][n][3]."""
    out, meas = [], []
    reached = np.zeros(len(b), dtype=bool)
    done = 0
    while done < max_steps and not reached.all():
        _, r = b.run(check_every, check_every, 0.0)
        out.append(r.copy())
        meas.append(np.array([measures(b[i]) for i in range(len(b))]))
        reached |= r <= stop_tol
        done += check_every
    return np.array(out), np.array(meas)


def first_crossing(hist, tol: float, check_every: int):
    """Steps at which each instance's residual first drops to ``tol`` (NaN if
    it never does)."""
    out = np.full(hist.shape[1], np.nan)
    for i in range(hist.shape[1]):
        k = np.nonzero(hist[:, i] <= tol)[0]
        if k.size:
            out[i] = (k[0] + 1) * check_every
    return out


# the equilibrium gate: contact angle within 0.5 degrees, area and volume
# within 0.1 % of the reference equilibrium
GATE = (0.5, 1e-3, 1e-3)


def within_gate(m, ref) -> np.ndarray:
    """Whether measures m (..., 3) lie within GATE of the reference ref."""
    m, ref = np.asarray(m), np.asarray(ref)
    return ((np.abs(m[..., 0] - ref[..., 0]) <= GATE[0]) & (np.abs(m[..., 1] / ref[..., 1] - 1) <= GATE[1]) &
            (np.abs(m[..., 2] / ref[..., 2] - 1) <= GATE[2]))


def settled(meas, ref, check_every: int):
    """Steps from which each instance stays within GATE of its reference for
    every later check (NaN if the last check is outside)."""
    ok = within_gate(meas, ref[None])  # [checks][n]
    out = np.full(ok.shape[1], np.nan)
    for i in range(ok.shape[1]):
        if not ok[-1, i]:
            continue
        bad = np.nonzero(~ok[:, i])[0]
        out[i] = ((bad[-1] + 2) if bad.size else 1) * check_every
    return out


def compare(net: WarmStartNet, wls, wls_learned=None, max_steps: int = 8000, check_every: int = 250,
            tols=(1e-4, 5e-5), ref_steps: int = None):
    """Relaxation of the instances from their plain start (FP32, for
    ``ref_steps`` steps, default max_steps) and from the learned start
    (instances ``wls_learned``, default the same; ``max_steps`` steps), each
    set as one batch, with the equilibrium gate: the reference equilibrium of
    an instance is the plain run's last state.  Reported per tolerance: the
    first residual crossing, counted only where the learned state there is
    within GATE of the reference; and the steps from which each run's shape
    stays within GATE of the reference (time to the equilibrium shape: a run
    counts once it stays within the gate until its end).  Also the wall time
    of each relaxation and of the warm-start calls."""
    import time
    import torch
    out = {}
    for name, ws_, learned in (("plain", wls, False), ("learned", wls_learned or wls, True)):
        b = Batch(ws_, device=net.device).init()
        torch.cuda.synchronize(net.device)
        t0 = time.perf_counter()
        if learned:
            for i, wl in enumerate(ws_):
                net.warm_start(b[i], features(wl))
        torch.cuda.synchronize(net.device)
        t_ws = time.perf_counter() - t0
        n_steps = (ref_steps or max_steps) if not learned else max_steps
        h, m = histories(b, n_steps, check_every, 0.0)
        torch.cuda.synchronize(net.device)
        out[name] = {"history": h, "measures": m, "wall_s": time.perf_counter() - t0, "warm_start_s": t_ws,
                     "first": {t: first_crossing(h, t, check_every) for t in tols}}
        del b
        torch.cuda.empty_cache()
    ref = out["plain"]["measures"][-1]  # [n][3]
    for name in ("plain", "learned"):
        m = out[name]["measures"]
        out[name]["shape_steps"] = settled(m, ref, check_every)
        for t in tols:
            # measures at the first residual crossing, and the gate there
            f = out[name]["first"][t]
            at = np.full((len(f), 3), np.nan)
            for i, v in enumerate(f):
                if np.isfinite(v):
                    at[i] = m[int(v) // check_every - 1, i]
            out[name].setdefault("gate", {})[t] = within_gate(at, ref)
            out[name].setdefault("dev", {})[t] = np.stack([np.abs(at[:, 0] - ref[:, 0]),
                                                           np.abs(at[:, 1] / ref[:, 1] - 1),
                                                           np.abs(at[:, 2] / ref[:, 2] - 1)], 1)

    def ratios(p, l):
        ok = np.isfinite(p) & np.isfinite(l)
        return {"both": int(ok.sum()),
                "plain_median": float(np.nanmedian(p)) if np.isfinite(p).any() else None,
                "learned_median": float(np.nanmedian(l)) if np.isfinite(l).any() else None,
                "median": float(np.median(p[ok] / l[ok])) if ok.any() else None,
                "geomean": float(np.exp(np.mean(np.log(p[ok] / l[ok])))) if ok.any() else None}

    for t in tols:
        p, l = out["plain"]["first"][t], out["learned"]["first"][t].copy()
        g = out["learned"]["gate"][t]
        dev = out["learned"]["dev"][t]
        ungated = ratios(p, l.copy())
        l[~g] = np.nan  # a learned crossing counts only within the gate
        r = ratios(p, l)
        r["ungated"] = ungated  # the residual crossings alone, without the gate
        r["gated"] = int(g.sum())
        r["max_dev_angle_deg"] = float(np.nanmax(dev[:, 0])) if np.isfinite(dev[:, 0]).any() else None
        r["max_dev_area"] = float(np.nanmax(dev[:, 1])) if np.isfinite(dev[:, 1]).any() else None
        r["max_dev_volume"] = float(np.nanmax(dev[:, 2])) if np.isfinite(dev[:, 2]).any() else None
        # the same gate for the plain run at its own crossing: how far the
        # reference itself still is from the plain state at that time
        gp, dp = out["plain"]["gate"][t], out["plain"]["dev"][t]
        r["plain_gated"] = int(gp.sum())
        for j, k in enumerate(("angle_deg", "area", "volume")):
            col = dp[:, j]
            r[f"plain_max_dev_{k}"] = float(np.nanmax(col)) if np.isfinite(col).any() else None
            r[f"median_dev_{k}"] = float(np.nanmedian(dev[:, j])) if np.isfinite(dev[:, j]).any() else None
            r[f"plain_median_dev_{k}"] = float(np.nanmedian(col)) if np.isfinite(col).any() else None
        out[f"ratio_{t:g}"] = r
    out["ratio_shape"] = ratios(out["plain"]["shape_steps"], out["learned"]["shape_steps"])
    return out


def experiment(edge: int = 48, n_train: int = 128, n_test: int = 64, relax_steps: int = 15000,
               target_tol: float = 2e-5, max_steps: int = 8000, check_every: int = 250, tols=(1e-4, 5e-5),
               epochs: int = 150, batch: int = 8, lr: float = 1e-3, lam: float = 1.0, seed: int = 0,
               ref_steps: int = 20000, device="cuda:0", log=print):
    """Time to equilibrium from the plain and from the learned start.

    Training instances: sweep seeds 1000.., relaxed in FP32 to the residual
    ``target_tol`` (or ``relax_steps``); held-out instances: seeds 5000...
    The held-out instances relax from the plain start in FP32 and from the
    learned start in FP16 storage; reported are the first steps at which the
    residual drops to each tolerance, and the wall times.  Returns a dict."""
    import time
    import torch
    out = {"edge": edge, "n_train": n_train, "n_test": n_test, "target_tol": target_tol}
    net = WarmStartNet(edge, 16, 4, max_batch=batch, max_nodes=642, device=device)
    net.set_params(init_params(net, seed))
    t0 = time.perf_counter()
    parts = []
    for k in range(0, n_train, 64):
        wls = [instances(1, seed=1000 + k + j, edge=edge)[0] for j in range(min(64, n_train - k))]
        parts.append(dataset(net, wls, relax_steps, check_every=1000, tol=target_tol))
        log(f"relaxed {k + len(wls)} training instances, median steps {np.median(parts[-1]['steps']):.0f}")
    data = {key: (torch.cat([p[key] for p in parts]) if torch.is_tensor(parts[0][key])
                  else np.concatenate([p[key] for p in parts])) for key in parts[0]}
    out["data_s"] = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train(net, data, epochs, batch=batch, lr=lr, lam=lam, seed=seed)
    torch.cuda.synchronize()
    out["train_s"] = time.perf_counter() - t0
    out["train_steps"] = len(losses)
    out["loss_first"], out["loss_last"] = float(np.mean(losses[:5])), float(np.mean(losses[-20:]))
    log(f"trained {len(losses)} steps in {out['train_s']:.1f} s, loss {out['loss_first']:.3e} -> {out['loss_last']:.3e}")
    del data, parts
    torch.cuda.empty_cache()
    test = [instances(1, seed=5000 + j, edge=edge)[0] for j in range(n_test)]
    test16 = [instances(1, seed=5000 + j, edge=edge, storage="f16")[0] for j in range(n_test)]
    r = compare(net, test, test16, max_steps, check_every, tols, ref_steps=ref_steps)
    fin = lambda a: [None if not np.isfinite(v) else int(v) for v in a]  # noqa: E731
    for k in ("plain", "learned"):
        out[k] = {"wall_s": r[k]["wall_s"], "warm_start_s": r[k]["warm_start_s"],
                  "first": {f"{t:g}": fin(r[k]["first"][t]) for t in tols},
                  "shape_steps": fin(r[k]["shape_steps"])}
    for t in tols:
        out[f"ratio_{t:g}"] = r[f"ratio_{t:g}"]
        log(f"tol {t:g}: {r[f'ratio_{t:g}']}")
    out["ratio_shape"] = r["ratio_shape"]
    out["gate"] = {"angle_deg": GATE[0], "area_rel": GATE[1], "volume_rel": GATE[2],
                   "reference": "the plain FP32 run's last state"}
    log(f"time to the equilibrium shape: {r['ratio_shape']}")
    out["params"] = net.params()
    return out
