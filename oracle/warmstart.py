"""FP64 CPU reference of the learned warm start (TEST INFRASTRUCTURE ONLY:
used by ``tests/`` and ``bench.py``'s CPU baseline, never by the library).

The warm start maps the plain initial state of a capsule-on-interface run
(the undeformed capsule on the flat interface, Sec. 4 set-ups) and its
parameters to a guess of the equilibrium the lattice Boltzmann + immersed
boundary relaxation reaches: corrections of phi and psi on the lattice and
a displacement field whose values at the markers move them.  The paper has
no learned component; the network is this library's addition, defined here
in plain PyTorch CPU operations (conv3d, avg_pool3d, nearest upsampling),
which serve as library primitives.

Network (E^3 lattice, channels-last on the GPU, NCDHW here):
  input  x: 16 channels -- phi0, psi0, five broadcast normalised
            parameters, nine zero channels
  encoder level l = 0..3 (edge E / 2^l, c_l = c0 2^l channels):
            e_l = relu(conv3(relu(conv3(in_l)))),  in_0 = x,
            in_l = avgpool2(e_{l-1})
  decoder level l = 2..0: d_l = relu(conv3(relu(conv3([up2(d_{l+1}) | e_l])))),
            d_3 = e_3
  output y = conv1(d_0): 16 channels -- dphi, dpsi, displacement (3), 11 unused
  phi = phi0 + y0, psi = psi0 + y1, marker offset = trilinear(y2..4)(X0)
conv3: 3x3x3, stride 1, zero padding 1; weights W[tap][ci][co] with tap =
(kz*3 + ky)*3 + kx for the offset (kz-1, ky-1, kx-1); conv1: 1x1x1.  Every
conv has a bias.  Stored activations are rounded to bfloat16 when
``bf16=True`` (the GPU stores them so); arithmetic is FP64.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CIN = 16       # input channels (7 used)
COUT = 16      # output channels (5 used)
NFEAT = 5      # broadcast parameters


def layer_shapes(c0: int = 16, levels: int = 4):
    """(taps, ci, co) of every conv, in parameter order."""
    c = [c0 * 2 ** l for l in range(levels)]
    out = [(27, CIN, c[0]), (27, c[0], c[0])]
    for l in range(1, levels):
        out += [(27, c[l - 1], c[l]), (27, c[l], c[l])]
    for l in range(levels - 2, -1, -1):
        out += [(27, c[l + 1] + c[l], c[l]), (27, c[l], c[l])]
    out.append((1, c[0], COUT))
    return out


def n_params(c0: int = 16, levels: int = 4) -> int:
    return sum(t * ci * co + co for t, ci, co in layer_shapes(c0, levels))


def init_params(seed: int, c0: int = 16, levels: int = 4) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, zero output
    layer (the untrained network returns the plain start), float32."""
    rng = np.random.default_rng(seed)
    out = []
    shapes = layer_shapes(c0, levels)
    for k, (t, ci, co) in enumerate(shapes):
        if k == len(shapes) - 1:
            w = np.zeros(t * ci * co)
        else:
            w = rng.normal(0.0, np.sqrt(2.0 / (t * ci)), t * ci * co)
        out += [w, np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


def unpack(theta, c0: int = 16, levels: int = 4):
    """[(W[tap][ci][co], b[co])] views of a flat parameter vector."""
    out, o = [], 0
    for t, ci, co in layer_shapes(c0, levels):
        W = theta[o:o + t * ci * co].reshape(t, ci, co)
        o += t * ci * co
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    assert o == len(theta)
    return out


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64:
    the float32 value's low 16 bits are rounded away (IEEE binary32 layout)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


class _RoundBF16(torch.autograd.Function):
    """bf16 rounding of a stored activation; the gradient passes through."""

    @staticmethod
    def forward(ctx, x):
        return torch.from_numpy(round_bf16(x.detach().numpy()))

    @staticmethod
    def backward(ctx, g):
        return g


def _conv(x, W, b, taps):
    co = W.shape[2]
    k = 3 if taps == 27 else 1
    w = W.reshape(k, k, k, W.shape[1], co).permute(4, 3, 0, 1, 2)
    return F.conv3d(x, w, b, padding=k // 2)


def features(kappa, G, R, E):
    """The five broadcast inputs, normalised to about [-1, 1] over the sweep
    ranges kappa_i in [0.005, 0.03], G in [0.002, 0.05], R/E in [0.15, 0.25]."""
    k = np.asarray(kappa, dtype=np.float64)
    return np.array([(k[0] - 0.0175) / 0.0125, (k[1] - 0.0175) / 0.0125, (k[2] - 0.0175) / 0.0125,
                     (G - 0.026) / 0.024, (R / E - 0.2) / 0.05])


def make_input(phi0: np.ndarray, psi0: np.ndarray, feats: np.ndarray, E: int) -> np.ndarray:
    """Network input [CIN][E][E][E] from the plain-start fields (linear
    lattice order, index (z*E + y)*E + x) and the features."""
    x = np.zeros((CIN, E, E, E))
    x[0] = phi0.reshape(E, E, E)
    x[1] = psi0.reshape(E, E, E)
    for k in range(NFEAT):
        x[2 + k] = feats[k]
    return x


def trilinear(D, X):
    """Values of the fields D [3][E][E][E] at points X [n][3] (x, y, z in
    lattice units; grid points at integer coordinates), coordinates clamped
    to [0, E-1]."""
    E = D.shape[-1]
    Xc = torch.clamp(X, 0.0, E - 1.0)
    i0 = torch.clamp(torch.floor(Xc), 0, E - 2).long()
    f = Xc - i0.double()
    out = torch.zeros(X.shape[0], D.shape[0], dtype=D.dtype)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                     * (f[:, 2] if dz else 1 - f[:, 2]))
                v = D[:, i0[:, 2] + dz, i0[:, 1] + dy, i0[:, 0] + dx].T
                out = out + w[:, None] * v
    return out


def forward(theta, x, X0=None, bf16: bool = True, c0: int = 16, levels: int = 4):
    """Network output y [B][COUT][E][E][E] (FP64) for inputs x [B][CIN][E^3],
    and the marker offsets trilinear(y2..4)(X0[b]) when X0 (list of [n][3]) is
    given.  ``theta`` may be a torch tensor that requires grad."""
    if not torch.is_tensor(theta):
        theta = torch.from_numpy(np.asarray(theta, dtype=np.float64))
    x = torch.as_tensor(np.asarray(x, dtype=np.float64)) if not torch.is_tensor(x) else x
    rnd = _RoundBF16.apply if bf16 else (lambda t: t)
    P = unpack(theta, c0, levels)
    Wq = [(rnd(W) if bf16 else W, b) for W, b in P]
    h = rnd(x)
    enc = []
    k = 0
    for l in range(levels):
        if l > 0:
            h = rnd(F.avg_pool3d(h, 2))
        for _ in range(2):
            W, b = Wq[k]
            h = rnd(torch.relu(_conv(h, W, b, 27)))
            k += 1
        enc.append(h)
    d = enc[-1]
    for l in range(levels - 2, -1, -1):
        u = F.interpolate(d, scale_factor=2, mode="nearest")
        h = torch.cat([u, enc[l]], dim=1)
        for _ in range(2):
            W, b = Wq[k]
            h = rnd(torch.relu(_conv(h, W, b, 27)))
            k += 1
        d = h
    W, b = Wq[k]
    y = _conv(d, W, b, 1)
    offs = None
    if X0 is not None:
        offs = [trilinear(y[i, 2:5], torch.as_tensor(np.asarray(X0[i], dtype=np.float64)))
                for i in range(y.shape[0])]
    return y, offs


def loss(theta, x, dphi_t, dpsi_t, X0, off_t, lam: float = 1.0, bf16: bool = True, c0: int = 16,
         levels: int = 4):
    """L = mean over samples and cells of (y0 - dphi_t)^2 + (y1 - dpsi_t)^2,
    plus lam times the mean over samples, markers and axes of (offset -
    off_t)^2.  The targets are the equilibrium minus the plain start:
    dphi_t, dpsi_t [B][E^3]; off_t a list of [n][3]."""
    y, offs = forward(theta, x, X0, bf16, c0, levels)
    B = y.shape[0]
    tp = torch.as_tensor(np.asarray(dphi_t, dtype=np.float64)).reshape(y[:, 0].shape)
    ts = torch.as_tensor(np.asarray(dpsi_t, dtype=np.float64)).reshape(y[:, 1].shape)
    Lf = ((y[:, 0] - tp) ** 2 + (y[:, 1] - ts) ** 2).mean()
    Lx = sum(((offs[i] - torch.as_tensor(np.asarray(off_t[i], dtype=np.float64))) ** 2).sum()
             for i in range(B)) / sum(3 * len(o) for o in off_t)
    return Lf + lam * Lx


def grad(theta, *args, **kw) -> np.ndarray:
    """dL/dtheta by reverse-mode differentiation of ``loss`` (FP64)."""
    t = torch.from_numpy(np.asarray(theta, dtype=np.float64)).requires_grad_(True)
    L = loss(t, *args, **kw)
    L.backward()
    return t.grad.numpy().copy()


def adam(theta, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1) of float64 copies;
    returns (theta, m, v) after step t (t counts from 1)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def mass_projection(phi, psi, phi_ref, psi_ref):
    """Shift phi and psi uniformly so that their totals equal those of the
    reference (plain) state: the lattice Boltzmann update conserves them, so
    the equilibrium has the plain start's totals."""
    n = phi.size
    return phi + (phi_ref.sum() - phi.sum()) / n, psi + (psi_ref.sum() - psi.sum()) / n


def vertex_normals(X: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Unit angle-weighted pseudo-normals of a closed triangle mesh
    (Baerentzen and Aanaes 2005): per vertex the sum over its faces of the
    face's unit normal times the face angle at the vertex, normalised."""
    N = np.zeros_like(X)
    for f in F:
        p = X[f]
        fn = np.cross(p[1] - p[0], p[2] - p[0])
        fn /= np.linalg.norm(fn)
        for k in range(3):
            a, b = p[(k + 1) % 3] - p[k], p[(k + 2) % 3] - p[k]
            ang = np.arccos(np.clip(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)), -1.0, 1.0))
            N[f[k]] += ang * fn
    return N / np.linalg.norm(N, axis=1, keepdims=True)


def enclosed_volume(X: np.ndarray, F: np.ndarray) -> float:
    """Volume of the closed triangle mesh (X, F), counter-clockwise from
    outside, by the divergence theorem: sum over faces of a . (b x c) / 6."""
    a, b, c = X[F[:, 0]], X[F[:, 1]], X[F[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def warm_start_markers(y, X0, normals, F=None):
    """Markers of the warm start: D = trilinear(y2..4)(X0); X0 + T + ((D - T).n) n
    with T the mean of D over the markers and n the unit vertex normals; with
    the faces F, then scaled about the centroid by (V(X0) / V(X))^(1/3), so
    that the moved membrane encloses the plain start's volume (the method
    conserves the fluid inside)."""
    D = trilinear(torch.as_tensor(np.asarray(y, dtype=np.float64))[2:5],
                  torch.as_tensor(np.asarray(X0, dtype=np.float64))).numpy()
    T = D.mean(axis=0)
    r = np.einsum("ij,ij->i", D - T, normals)
    X = X0 + T + r[:, None] * normals
    if F is not None:
        s = (enclosed_volume(X0, F) / enclosed_volume(X, F)) ** (1.0 / 3.0)
        c = X.mean(axis=0)
        X = c + s * (X - c)
    return X


def warm_start_fields(y0, phi0, psi0, I_new, factors=False):
    """Fields of the warm start from the output y0 (the change of the phase
    indicator s = phi / (1 - psi)), the plain start and the profile I_new of
    the moved markers.  The method conserves the totals of psi and phi
    (Sec. 2, the advection-diffusion equations of C_m are in conservation
    form); the warm start restores the plain totals by moving the
    interfaces, not by shifting the bulk values away from the minimisers
    of the bulk free energy:
        psi = I_new + l_psi 4 I_new (1 - I_new),
        phi = (1 - psi)(s + l_phi (1 - s^2)_+),  s = s0 + y0,
    with l_psi, l_phi the factors that restore the totals (0 when their
    weights vanish everywhere), returned after the fields when `factors`."""
    w0 = 1.0 - psi0
    s0 = np.where(w0 > 1e-6, phi0 / np.where(w0 > 1e-6, w0, 1.0), 0.0)
    wpsi = 4.0 * I_new * (1.0 - I_new)
    l_psi = (psi0.sum() - I_new.sum()) / wpsi.sum() if wpsi.sum() > 1e-12 else 0.0
    psi = I_new + l_psi * wpsi
    s = s0 + y0
    w = 1.0 - psi
    wphi = np.maximum(0.0, 1.0 - s * s)
    den = (w * wphi).sum()
    l_phi = (phi0.sum() - (w * s).sum()) / den if den > 1e-12 else 0.0
    if factors:
        return w * (s + l_phi * wphi), psi, l_psi, l_phi
    return w * (s + l_phi * wphi), psi
