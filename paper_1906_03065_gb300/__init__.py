"""GB300 ternary free-energy lattice Boltzmann + immersed boundary library.

Python binding of the C ABI in ``include/tlb.h`` (``libtlb.so``).  It only
marshals arguments: every step of the method runs in the library's CUDA
kernels.  PyTorch supplies the device arena and the CUDA stream.

The shared library is loaded on first use; if it is missing (not built) or
no CUDA device is present the calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads  # noqa: F401  (seeded input generators)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtlb.so")
_lib = None

TLB_OK = 0
STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
FIELD = {"rho": 0, "phi": 1, "psi": 2, "C1": 3, "C2": 4, "C3": 5, "u": 6, "I": 7}


class TLBError(RuntimeError):
    pass


class _Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("wall_last", C.c_int), ("storage", C.c_int),
                ("tau", C.c_double), ("tau_phi", C.c_double), ("tau_psi", C.c_double),
                ("gamma_phi", C.c_double), ("gamma_psi", C.c_double), ("alpha", C.c_double),
                ("kappa", C.c_double * 3), ("kappa_c", C.c_double), ("dc", C.c_double),
                ("u0", C.c_double * 3), ("interface_pos", C.c_double), ("forcing", C.c_int),
                ("state", C.c_int), ("force_form", C.c_int)]


class _Mem(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_nodes", C.c_int), ("n_elems", C.c_int),
                ("X0", C.POINTER(C.c_double)), ("elems", C.POINTER(C.c_int)),
                ("ks", C.c_double), ("kb", C.c_double),
                ("skalak_G", C.c_double), ("skalak_C", C.c_double)]


class _Inst(C.Structure):
    _fields_ = [("params", _Params), ("mems", C.POINTER(_Mem)), ("n_mem", C.c_int)]


class _NetDesc(C.Structure):
    _fields_ = [("edge", C.c_int), ("base_channels", C.c_int), ("levels", C.c_int),
                ("max_batch", C.c_int), ("max_nodes", C.c_int)]


class Diag(C.Structure):
    _fields_ = [("step", C.c_long), ("mass", C.c_double * 3), ("umax", C.c_double),
                ("n_caps", C.c_int), ("area", C.c_double * 8), ("volume", C.c_double * 8)]


class Profile(C.Structure):
    _fields_ = [("steps", C.c_long), ("ms_moments", C.c_double), ("ms_ibm", C.c_double),
                ("ms_collide", C.c_double), ("ms_interp", C.c_double), ("launches_per_step", C.c_long)]


def lib():
    """Load libtlb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TLBError(f"{LIB_PATH} is missing: run paper_1906_03065_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        vp, dp, sz = C.c_void_p, C.POINTER(C.c_double), C.c_size_t
        L.tlb_state_bytes.argtypes = [C.POINTER(_Params), C.POINTER(_Mem), C.c_int, C.POINTER(sz)]
        L.tlb_create.argtypes = [C.POINTER(_Params), C.POINTER(_Mem), C.c_int, vp, sz, vp, C.POINTER(vp)]
        L.tlb_init_fields.argtypes = [vp, dp, dp]
        L.tlb_step.argtypes = [vp, C.c_long]
        L.tlb_read_field.argtypes = [vp, C.c_int, dp, sz]
        L.tlb_read_nodes.argtypes = [vp, C.c_int, dp, sz]
        L.tlb_write_nodes.argtypes = [vp, C.c_int, dp, sz]
        L.tlb_read_populations.argtypes = [vp, dp, sz]
        L.tlb_write_populations.argtypes = [vp, dp, sz]
        L.tlb_diagnostics.argtypes = [vp, C.POINTER(Diag)]
        L.tlb_diagnostics_static.argtypes = [vp, C.POINTER(Diag)]
        L.tlb_diagnostics_static.restype = C.c_int
        L.tlb_profile_steps.argtypes = [vp, C.c_long, C.POINTER(Profile)]
        L.tlb_profile_steps.restype = C.c_int
        L.tlb_autotune.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.tlb_autotune.restype = C.c_int
        L.tlb_last_launch_count.argtypes = [vp]
        L.tlb_last_launch_count.restype = C.c_long
        L.tlb_run.argtypes = [vp, C.c_long, C.c_long, C.c_double, C.POINTER(C.c_long), dp]
        L.tlb_save.argtypes = [vp, vp, C.POINTER(sz)]
        L.tlb_load.argtypes = [vp, vp, sz]
        for n in ("tlb_run", "tlb_save", "tlb_load"):
            getattr(L, n).restype = C.c_int
        L.tlb_set_tile.argtypes = [vp, C.c_int, C.c_int]
        L.tlb_set_tile.restype = C.c_int
        L.tlb_set_graphs.argtypes = [vp, C.c_int]
        L.tlb_set_graphs.restype = C.c_int
        L.tlb_residual.argtypes = [vp, dp]
        L.tlb_residual.restype = C.c_int
        L.tlb_contact_angle.argtypes = [vp, dp, sz]
        L.tlb_contact_angle.restype = C.c_int
        ip, lp = C.POINTER(C.c_int), C.POINTER(C.c_long)
        L.tlb_batch_state_bytes.argtypes = [C.POINTER(_Inst), C.c_int, C.POINTER(sz)]
        L.tlb_batch_create.argtypes = [C.POINTER(_Inst), C.c_int, vp, sz, vp, C.POINTER(vp)]
        L.tlb_batch_instance.argtypes = [vp, C.c_int, C.POINTER(vp)]
        L.tlb_batch_set_active.argtypes = [vp, ip]
        L.tlb_batch_step.argtypes = [vp, C.c_long]
        L.tlb_batch_run.argtypes = [vp, C.c_long, C.c_long, C.c_double, lp, dp]
        L.tlb_batch_autotune.argtypes = [vp, ip, ip]
        for n in ("tlb_batch_state_bytes", "tlb_batch_create", "tlb_batch_instance", "tlb_batch_set_active",
                  "tlb_batch_step", "tlb_batch_run", "tlb_batch_autotune"):
            getattr(L, n).restype = C.c_int
        L.tlb_batch_profile_steps.argtypes = [vp, C.c_long, dp]
        L.tlb_batch_profile_steps.restype = C.c_int
        L.tlb_batch_launch_count.argtypes = [vp]
        L.tlb_batch_launch_count.restype = C.c_long
        L.tlb_batch_destroy.argtypes = [vp]
        fp = C.POINTER(C.c_float)
        nd = C.POINTER(_NetDesc)
        L.tlb_net_param_count.argtypes = [nd, C.POINTER(sz)]
        L.tlb_net_state_bytes.argtypes = [nd, C.POINTER(sz)]
        L.tlb_net_create.argtypes = [nd, vp, sz, vp, C.POINTER(vp)]
        L.tlb_net_set_params.argtypes = [vp, fp, sz]
        L.tlb_net_get_params.argtypes = [vp, fp, sz]
        L.tlb_net_get_grads.argtypes = [vp, fp, sz]
        L.tlb_net_input.argtypes = [vp, vp, dp, vp]
        L.tlb_net_forward.argtypes = [vp, vp, C.c_int, vp]
        L.tlb_net_train_step.argtypes = [vp, vp, vp, vp, vp, vp, ip, C.c_int, C.c_double, C.c_double, C.c_int, dp]
        L.tlb_net_warm_start.argtypes = [vp, vp, dp]
        for n in ("tlb_net_param_count", "tlb_net_state_bytes", "tlb_net_create", "tlb_net_set_params",
                  "tlb_net_get_params", "tlb_net_get_grads", "tlb_net_input", "tlb_net_forward",
                  "tlb_net_train_step", "tlb_net_warm_start"):
            getattr(L, n).restype = C.c_int
        L.tlb_net_launch_count.argtypes = [vp]
        L.tlb_net_launch_count.restype = C.c_long
        L.tlb_net_set_tcgen05.argtypes = [vp, C.c_int]
        L.tlb_net_set_tcgen05.restype = C.c_int
        L.tlb_net_status.argtypes = [vp, C.POINTER(C.c_uint)]
        L.tlb_net_status.restype = C.c_int
        L.tlb_net_destroy.argtypes = [vp]
        L.tlb_destroy.argtypes = [vp]
        L.tlb_last_error.restype = C.c_char_p
        for n in ("tlb_state_bytes", "tlb_create", "tlb_init_fields", "tlb_step", "tlb_read_field",
                  "tlb_read_nodes", "tlb_write_nodes", "tlb_read_populations",
                  "tlb_write_populations", "tlb_diagnostics"):
            getattr(L, n).restype = C.c_int
        _lib = L
    return _lib


def _check(st):
    if st != TLB_OK:
        msg = lib().tlb_last_error().decode()
        raise TLBError(f"tlb status {st}: {msg}")


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(p) -> _Params:
    """``p`` is a ``workloads.Params``."""
    cp = _Params()
    cp.dim, cp.nx, cp.ny, cp.nz = p.dim, p.nx, p.ny, (p.nz if p.dim == 3 else 1)
    cp.wall_last = p.wall_last
    cp.storage = STORAGE[p.storage]
    cp.tau, cp.tau_phi, cp.tau_psi = p.tau, p.tau_phi, p.tau_psi
    cp.gamma_phi, cp.gamma_psi, cp.alpha = p.gamma_phi, p.gamma_psi, p.alpha
    cp.kappa[0], cp.kappa[1], cp.kappa[2] = p.kappa1, p.kappa2, p.kappa3
    cp.kappa_c, cp.dc = p.kappa_c, p.dc
    for k in range(3):
        cp.u0[k] = p.u0[k]
    cp.interface_pos = p.interface_pos
    cp.forcing = {"edm": 0, "guo": 1}[getattr(p, "forcing", "edm")]
    cp.state = {"populations": 0, "moments": 1}[getattr(p, "state", "populations")]
    cp.force_form = {"potential": 0, "pressure_tensor": 1}[getattr(p, "force_form", "potential")]
    return cp


def _marshal_membranes(wl, keep):
    """tlb_membrane_desc array of a workload; arrays it points to go to ``keep``."""
    mems = (_Mem * max(1, len(wl.membranes)))()
    for i, m in enumerate(wl.membranes):
        X = np.ascontiguousarray(m.X, dtype=np.float64)
        E = np.ascontiguousarray(m.elems if m.elems is not None else np.zeros((1, 3)), dtype=np.int32)
        keep += [X, E]
        mems[i].kind = m.kind
        mems[i].n_nodes = X.shape[0]
        mems[i].n_elems = E.shape[0] if m.kind == 1 else 0
        mems[i].X0 = _dp(X)
        mems[i].elems = E.ctypes.data_as(C.POINTER(C.c_int)) if m.kind == 1 else None
        mems[i].ks, mems[i].kb = m.ks, m.kb
        mems[i].skalak_G, mems[i].skalak_C = m.G, m.C
    return mems


class Simulation:
    """One lattice with its membranes on the current CUDA device.

    ``wl`` is a ``workloads.Workload``.  The arena is a torch uint8 tensor on
    ``device``; the stream is torch's current stream unless given.
    """

    def __init__(self, wl, device="cuda:0", stream=None, _handle=None, _owner=None):
        self.wl = wl
        p = wl.params
        self.p = p
        self.n_mem = len(wl.membranes)
        self.nn = [m.X.shape[0] for m in wl.membranes]
        self.N = p.nx * p.ny * (p.nz if p.dim == 3 else 1)
        self.Q = 19 if p.dim == 3 else 9
        if _handle is not None:  # instance of a Batch: borrowed handle
            self.h = _handle
            self._owner = _owner
            return
        self._owner = None
        import torch
        L = lib()
        self._cp = make_params(p)
        self._keep = []
        mems = _marshal_membranes(wl, self._keep)
        self._mems = mems
        nbytes = C.c_size_t(0)
        _check(L.tlb_state_bytes(C.byref(self._cp), mems, self.n_mem, C.byref(nbytes)))
        self.nbytes = nbytes.value
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.arena = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            base = self.arena.data_ptr()
            aligned = (base + 255) // 256 * 256
            h = C.c_void_p()
            _check(L.tlb_create(C.byref(self._cp), mems, self.n_mem, C.c_void_p(aligned),
                                C.c_size_t(self.nbytes), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def __del__(self):
        try:
            if getattr(self, "_owner", None) is None and getattr(self, "h", None) is not None and self.h.value:
                lib().tlb_destroy(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def shape(self):
        p = self.p
        return (p.nz, p.ny, p.nx) if p.dim == 3 else (p.ny, p.nx)

    def init(self, Cf=None, u=None):
        cf = None if Cf is None else np.ascontiguousarray(Cf, dtype=np.float64)
        uf = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        _check(lib().tlb_init_fields(self.h, None if cf is None else _dp(cf), None if uf is None else _dp(uf)))
        return self

    def step(self, n: int = 1):
        _check(lib().tlb_step(self.h, int(n)))

    def autotune(self):
        """Pick the collide tile shape and z chunk by timing; returns them."""
        v, z = C.c_int(0), C.c_int(0)
        _check(lib().tlb_autotune(self.h, C.byref(v), C.byref(z)))
        return v.value, z.value

    def run(self, max_steps: int, check_every: int = 100, tol: float = 1e-8):
        """Step until the residual reaches ``tol`` (checked every
        ``check_every`` steps) or ``max_steps``; returns (t, residual)."""
        t, r = C.c_long(0), C.c_double(0)
        _check(lib().tlb_run(self.h, int(max_steps), int(check_every), float(tol), C.byref(t), C.byref(r)))
        return t.value, r.value

    def save(self) -> np.ndarray:
        """Checkpoint (host bytes) from which ``load`` resumes exactly."""
        n = C.c_size_t(0)
        _check(lib().tlb_save(self.h, None, C.byref(n)))
        blob = np.empty(n.value, dtype=np.uint8)
        _check(lib().tlb_save(self.h, C.c_void_p(blob.ctypes.data), C.byref(n)))
        return blob

    def load(self, blob):
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(lib().tlb_load(self.h, C.c_void_p(b.ctypes.data), b.size))
        return self

    def set_tile(self, variant: int, z_chunk: int):
        _check(lib().tlb_set_tile(self.h, int(variant), int(z_chunk)))

    def set_graphs(self, on: bool):
        _check(lib().tlb_set_graphs(self.h, int(bool(on))))

    def launches(self) -> int:
        return lib().tlb_last_launch_count(self.h)

    def field(self, name: str, out=None) -> np.ndarray:
        """A field as doubles (``u``: shape (3, N)); ``out`` may supply the
        host buffer (e.g. pinned memory) of N (3 N) contiguous doubles."""
        n = self.N * (3 if name == "u" else 1)
        if out is None:
            out = np.empty(n)
        elif out.dtype != np.float64 or out.size != n or not out.flags.c_contiguous:
            raise TLBError(f"field: out must hold {n} contiguous doubles")
        _check(lib().tlb_read_field(self.h, FIELD[name], _dp(out), n))
        return out.reshape(3, self.N) if name == "u" else out.reshape(-1)

    def nodes(self, m: int = 0) -> np.ndarray:
        out = np.zeros(3 * self.nn[m])
        _check(lib().tlb_read_nodes(self.h, m, _dp(out), out.size))
        return out.reshape(-1, 3)

    def set_nodes(self, m: int, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        _check(lib().tlb_write_nodes(self.h, m, _dp(X), X.size))

    def pops(self) -> np.ndarray:
        out = np.zeros(3 * self.Q * self.N)
        _check(lib().tlb_read_populations(self.h, _dp(out), out.size))
        return out.reshape(3, self.Q, self.N)

    def set_pops(self, P):
        P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1)
        _check(lib().tlb_write_populations(self.h, _dp(P), P.size))

    def profile(self, n: int) -> Profile:
        pr = Profile()
        _check(lib().tlb_profile_steps(self.h, int(n), C.byref(pr)))
        return pr

    def diagnostics(self) -> Diag:
        d = Diag()
        _check(lib().tlb_diagnostics(self.h, C.byref(d)))
        return d

    def contact_angle(self) -> np.ndarray:
        """Per capsule [mean, min, max angle in degrees, contact points] of
        the membrane with the phi = 0 interface (see tlb_contact_angle)."""
        out = np.zeros(4 * max(1, len(self.nn)))
        _check(lib().tlb_contact_angle(self.h, _dp(out), out.size))
        return out.reshape(-1, 4)[:len(self.nn)]

    def residual(self) -> np.ndarray:
        """[max |d phi|, max |d psi|, max |d X|, residual] since the last call
        (or init); see tlb_residual."""
        out = np.zeros(4)
        _check(lib().tlb_residual(self.h, _dp(out)))
        return out

    def diagnostics_static(self) -> Diag:
        """Diagnostics with the library's fixed scratch array (no device
        memory from the caller; see tlb_diagnostics_static in tlb.h)."""
        d = Diag()
        _check(lib().tlb_diagnostics_static(self.h, C.byref(d)))
        return d


class Batch:
    """Independent lattices of one dim and storage stepped together (one
    persistent launch per phase, graph-captured).  ``wls`` is a list of
    ``workloads.Workload``; ``batch[i]`` is instance i as a Simulation whose
    handle the batch owns."""

    def __init__(self, wls, device="cuda:0", stream=None):
        import torch
        L = lib()
        self.wls = list(wls)
        n = len(self.wls)
        self._keep = []
        descs = (_Inst * n)()
        for i, wl in enumerate(self.wls):
            descs[i].params = make_params(wl.params)
            mems = _marshal_membranes(wl, self._keep)
            self._keep.append(mems)
            descs[i].mems = C.cast(mems, C.POINTER(_Mem))
            descs[i].n_mem = len(wl.membranes)
        self._descs = descs
        nbytes = C.c_size_t(0)
        _check(L.tlb_batch_state_bytes(descs, n, C.byref(nbytes)))
        self.nbytes = nbytes.value
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.arena = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            aligned = (self.arena.data_ptr() + 255) // 256 * 256
            h = C.c_void_p()
            _check(L.tlb_batch_create(descs, n, C.c_void_p(aligned), C.c_size_t(self.nbytes),
                                      C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self._handles = []
        for i in range(n):
            ih = C.c_void_p()
            _check(L.tlb_batch_instance(self.h, i, C.byref(ih)))
            self._handles.append(ih)
        self.cells = sum(wl.params.ncells for wl in self.wls)

    def __len__(self):
        return len(self.wls)

    def __getitem__(self, i) -> Simulation:
        """Instance i (the view keeps the batch alive)."""
        return Simulation(self.wls[i], _handle=self._handles[i], _owner=self)

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                lib().tlb_batch_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def init(self):
        """Default initial state of every instance (as Simulation.init())."""
        for i in range(len(self)):
            self[i].init()
        return self

    def set_active(self, flags):
        f = np.ascontiguousarray(np.asarray(flags, dtype=np.int32))
        _check(lib().tlb_batch_set_active(self.h, f.ctypes.data_as(C.POINTER(C.c_int))))

    def step(self, n: int = 1):
        _check(lib().tlb_batch_step(self.h, int(n)))

    def run(self, max_steps: int, check_every: int = 100, tol: float = 1e-8):
        """Run to residual; returns (steps_done, residual) per instance."""
        steps = np.zeros(len(self), dtype=np.int64)
        res = np.zeros(len(self))
        _check(lib().tlb_batch_run(self.h, int(max_steps), int(check_every), float(tol),
                                   steps.ctypes.data_as(C.POINTER(C.c_long)), _dp(res)))
        return steps, res

    def autotune(self):
        v, z = C.c_int(0), C.c_int(0)
        _check(lib().tlb_batch_autotune(self.h, C.byref(v), C.byref(z)))
        return v.value, z.value

    def launches(self) -> int:
        return lib().tlb_batch_launch_count(self.h)

    PHASES = ("moments_geometry", "forces_scatter", "band", "spread_fill", "collide", "interp")

    def profile(self, n: int) -> dict:
        """Device ms per step of each phase over n steps (tlb_batch_profile_steps)."""
        ms = np.zeros(6)
        _check(lib().tlb_batch_profile_steps(self.h, int(n), _dp(ms)))
        return {k: v / max(n, 1) for k, v in zip(self.PHASES, ms)}


class WarmStartNet:
    """The warm-start encoder-decoder of tlb.h on one GPU: parameters, input
    construction, forward, training steps and the warm start of a context.
    Tensors are torch tensors on the net's device (x: bf16 [B, E^3, 16];
    targets fp32)."""

    def __init__(self, edge: int, base_channels: int = 16, levels: int = 4, max_batch: int = 8,
                 max_nodes: int = 0, device="cuda:0", stream=None):
        import torch
        L = lib()
        self.desc = _NetDesc(edge, base_channels, levels, max_batch, max_nodes)
        n = C.c_size_t(0)
        _check(L.tlb_net_param_count(C.byref(self.desc), C.byref(n)))
        self.n_params = n.value
        b = C.c_size_t(0)
        _check(L.tlb_net_state_bytes(C.byref(self.desc), C.byref(b)))
        self.nbytes = b.value
        self.edge, self.max_batch, self.max_nodes = edge, max_batch, max_nodes
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.arena = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            aligned = (self.arena.data_ptr() + 255) // 256 * 256
            h = C.c_void_p()
            _check(L.tlb_net_create(C.byref(self.desc), C.c_void_p(aligned), C.c_size_t(self.nbytes),
                                    C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                lib().tlb_net_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib().tlb_net_set_params(self.h, t.ctypes.data_as(C.POINTER(C.c_float)), t.size))

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().tlb_net_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), out.size))
        return out

    def grads(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().tlb_net_get_grads(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), out.size))
        return out

    def input(self, sim, feats, out=None):
        """Input tensor of a freshly initialised Simulation (plain start)."""
        import torch
        V = self.edge ** 3
        x = out if out is not None else torch.empty((V, 16), dtype=torch.bfloat16, device=self.device)
        f = np.ascontiguousarray(feats, dtype=np.float64)
        _check(lib().tlb_net_input(self.h, sim.h, _dp(f), C.c_void_p(x.data_ptr())))
        return x

    def forward(self, x):
        import torch
        B = x.shape[0] if x.dim() == 3 else 1
        y = torch.empty((B, self.edge ** 3, 16), dtype=torch.float32, device=self.device)
        _check(lib().tlb_net_forward(self.h, C.c_void_p(x.data_ptr()), B, C.c_void_p(y.data_ptr())))
        return y

    def train_step(self, x, dphi, dpsi, X0=None, off=None, n_nodes=None, lam: float = 1.0,
                   lr: float = 1e-3, update: bool = True) -> float:
        B = x.shape[0] if x.dim() == 3 else 1
        nn = None
        if n_nodes is not None:
            nn = np.ascontiguousarray(np.asarray(n_nodes, dtype=np.int32))
        loss = C.c_double(0)
        vp = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        _check(lib().tlb_net_train_step(self.h, vp(x), vp(dphi), vp(dpsi), vp(X0), vp(off),
                                        nn.ctypes.data_as(C.POINTER(C.c_int)) if nn is not None else None,
                                        B, float(lam), float(lr), int(bool(update)), C.byref(loss)))
        return loss.value

    def warm_start(self, sim, feats):
        """Replace the plain initial state of ``sim`` by the network's guess."""
        f = np.ascontiguousarray(feats, dtype=np.float64)
        _check(lib().tlb_net_warm_start(self.h, sim.h, _dp(f)))

    def set_tcgen05(self, mode: int):
        """2: tcgen05 fed by TMA (default), 1: tcgen05 with cp.async staging, 0: mma.sync."""
        _check(lib().tlb_net_set_tcgen05(self.h, int(mode)))

    def status(self) -> int:
        st = C.c_uint(0)
        _check(lib().tlb_net_status(self.h, C.byref(st)))
        return st.value

    def launches(self) -> int:
        return lib().tlb_net_launch_count(self.h)
