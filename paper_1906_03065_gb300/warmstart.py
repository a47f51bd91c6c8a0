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


def instances(n: int, seed: int, edge: int = 48, storage: str = "f32"):
    """``n`` sweep instances of one lattice edge (workloads.sweep_3d with a
    single edge, so every sample has the network's lattice)."""
    return W.sweep_3d(n, seed=seed, storage=storage, edges=(edge,))


def dataset(net: WarmStartNet, wls, max_steps: int, check_every: int = 200, tol: float = 1e-7):
    """Training tensors (on the net's device) of the instances ``wls``: the
    inputs of their plain starts, and the equilibrium minus the plain start
    (fields and marker offsets) after relaxing them together as a batch to
    the residual ``tol`` (or ``max_steps``).  Returns a dict with x, dphi,
    dpsi, X0, off, n_nodes, steps, residual."""
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
        dphi[i] = s.field("phi") - phi0[i]
        dpsi[i] = s.field("psi") - psi0[i]
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


def compare(net: WarmStartNet, wls, max_steps: int, check_every: int = 200, tol: float = 1e-7):
    """Relaxation of every instance from its plain start and from the learned
    start, side by side in one batch (instances 0..n-1 plain, n..2n-1
    learned).  Returns steps and final residual of each, and the wall time of
    the warm-start calls (s)."""
    import time
    import torch
    n = len(wls)
    b = Batch(list(wls) + list(wls), device=net.device).init()
    torch.cuda.synchronize(net.device)
    t0 = time.perf_counter()
    for i, wl in enumerate(wls):
        net.warm_start(b[n + i], features(wl))
    torch.cuda.synchronize(net.device)
    t_ws = time.perf_counter() - t0
    steps, res = b.run(max_steps, check_every, tol)
    return {"plain_steps": steps[:n], "learned_steps": steps[n:], "plain_residual": res[:n],
            "learned_residual": res[n:], "warm_start_s": t_ws, "batch": b}
