"""FP64 CPU oracle of the ternary LB + IBM step (ctypes binding).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never loads it.
It shares no code with the CUDA path; the only common module is the seeded
input generator ``paper_1906_03065_gb300.workloads`` (geometry and parameters,
no arithmetic of the method).

The C++ source is ``oracle/tlb_oracle.cpp``; each function there cites the
passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tlb_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libtlb_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP, -O2, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("wall_last", C.c_int), ("pad", C.c_int),
                ("tau", C.c_double), ("tau_phi", C.c_double), ("tau_psi", C.c_double),
                ("gamma_phi", C.c_double), ("gamma_psi", C.c_double), ("alpha", C.c_double),
                ("kappa1", C.c_double), ("kappa2", C.c_double), ("kappa3", C.c_double),
                ("kappa_c", C.c_double), ("dc", C.c_double),
                ("u0x", C.c_double), ("u0y", C.c_double), ("u0z", C.c_double),
                ("interface_pos", C.c_double), ("storage", C.c_int), ("forcing", C.c_int),
                ("force_form", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(_Params)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_set_threads.restype = C.c_int
        L.or_Q.argtypes = [C.c_void_p]
        L.or_lattice.argtypes = [C.c_void_p, C.POINTER(C.c_int), dp]
        L.or_add_membrane.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.c_int, C.POINTER(C.c_int),
                                      C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_add_membrane.restype = C.c_int
        L.or_init.argtypes = [C.c_void_p, dp, dp]
        L.or_step.argtypes = [C.c_void_p, C.c_int]
        L.or_time.argtypes = [C.c_void_p]
        L.or_time.restype = C.c_long
        for n in ("or_get_pops", "or_set_pops"):
            getattr(L, n).argtypes = [C.c_void_p, dp]
        L.or_get_nodes.argtypes = [C.c_void_p, C.c_int, dp]
        L.or_set_nodes.argtypes = [C.c_void_p, C.c_int, dp]
        L.or_get_field.argtypes = [C.c_void_p, C.c_int, dp]
        L.or_round.argtypes = [C.c_double, C.c_int, C.c_int, C.c_double]
        L.or_round.restype = C.c_double
        L.or_peskin.argtypes = [C.c_double]
        L.or_peskin.restype = C.c_double
        L.or_mem_energy.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        L.or_mem_energy.restype = C.c_double
        L.or_mem_force.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, dp]
        L.or_iprofile.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_iprofile.restype = C.c_long
        L.or_coupling.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_coupling.restype = C.c_double
        L.or_potentials.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp, dp]
        L.or_spread.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_interp.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        L.or_masses.argtypes = [C.c_void_p, dp]
        L.or_grad_field.argtypes = [C.c_void_p, dp, dp]
        L.or_lap_field.argtypes = [C.c_void_p, dp, dp]
        L.or_force_fe.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        L.or_bulk_pressure.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double]
        L.or_bulk_pressure.restype = C.c_double
        L.or_capsule_measures.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_contact_angle.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        L.or_contact_angle.restype = C.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


STORAGE_CODE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}

FORCING_CODE = {"edm": 0, "guo": 1}
FORCE_FORM_CODE = {"potential": 0, "pressure_tensor": 1}
FIELDS = {"rho": 0, "phi": 1, "psi": 2, "ux": 3, "uy": 4, "uz": 5, "C1": 6, "C2": 7,
          "C3": 8, "I": 9, "Fx": 10, "Fy": 11, "Fz": 12, "fibx": 13, "fiby": 14,
          "fibz": 15, "mu_rho": 16, "mu_phi": 17, "mu_psi": 18}


def set_threads(n: int = 0) -> int:
    return lib().or_set_threads(int(n))


class Oracle:
    """One oracle simulation.  ``wl`` is a ``workloads.Workload``."""

    def __init__(self, wl, init: bool = True, Cf=None, u=None, emulate_storage: bool = False):
        from paper_1906_03065_gb300.workloads import MEM_RING2D
        L = lib()
        p = wl.params
        self.p = p
        cp = _Params(p.dim, p.nx, p.ny, p.nz if p.dim == 3 else 1, p.wall_last, 0,
                     p.tau, p.tau_phi, p.tau_psi, p.gamma_phi, p.gamma_psi, p.alpha,
                     p.kappa1, p.kappa2, p.kappa3, p.kappa_c, p.dc,
                     p.u0[0], p.u0[1], p.u0[2], p.interface_pos,
                     STORAGE_CODE[p.storage] if emulate_storage else 0,
                     FORCING_CODE[getattr(p, "forcing", "edm")],
                     FORCE_FORM_CODE[getattr(p, "force_form", "potential")])
        self._cp = cp
        self.h = L.or_create(C.byref(cp))
        self.N = p.nx * p.ny * (p.nz if p.dim == 3 else 1)
        self.Q = L.or_Q(self.h)
        self.nn = []
        for m in wl.membranes:
            X = np.ascontiguousarray(m.X, dtype=np.float64)
            if m.kind == MEM_RING2D:
                E = np.zeros(1, dtype=np.int32)
                ne = X.shape[0]
            else:
                E = np.ascontiguousarray(m.elems, dtype=np.int32)
                ne = E.shape[0]
            L.or_add_membrane(self.h, m.kind, X.shape[0], _dp(X), ne,
                              E.ctypes.data_as(C.POINTER(C.c_int)), m.ks, m.kb, m.G, m.C)
            self.nn.append(X.shape[0])
        if init:
            self.init(Cf, u)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().or_destroy(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def shape(self):
        p = self.p
        return (p.nz, p.ny, p.nx) if p.dim == 3 else (p.ny, p.nx)

    def lattice(self):
        c = np.zeros(3 * self.Q, dtype=np.int32)
        w = np.zeros(self.Q)
        lib().or_lattice(self.h, c.ctypes.data_as(C.POINTER(C.c_int)), _dp(w))
        return c.reshape(self.Q, 3), w

    def init(self, Cf=None, u=None):
        cptr = None if Cf is None else _dp(np.ascontiguousarray(Cf, dtype=np.float64))
        uptr = None if u is None else _dp(np.ascontiguousarray(u, dtype=np.float64))
        self._keep = (Cf, u)
        if Cf is not None:
            self._c_arr = np.ascontiguousarray(Cf, dtype=np.float64)
            cptr = _dp(self._c_arr)
        if u is not None:
            self._u_arr = np.ascontiguousarray(u, dtype=np.float64)
            uptr = _dp(self._u_arr)
        lib().or_init(self.h, cptr, uptr)
        self._res_ref = self._res_state()

    def step(self, n: int = 1):
        lib().or_step(self.h, int(n))

    @property
    def t(self):
        return lib().or_time(self.h)

    def pops(self) -> np.ndarray:
        out = np.zeros(3 * self.Q * self.N)
        lib().or_get_pops(self.h, _dp(out))
        return out.reshape(3, self.Q, self.N)

    def set_pops(self, P: np.ndarray):
        P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1)
        lib().or_set_pops(self.h, _dp(P))

    def nodes(self, m: int = 0) -> np.ndarray:
        out = np.zeros(3 * self.nn[m])
        lib().or_get_nodes(self.h, m, _dp(out))
        return out.reshape(-1, 3)

    def set_nodes(self, m: int, X: np.ndarray):
        X = np.ascontiguousarray(X, dtype=np.float64)
        lib().or_set_nodes(self.h, m, _dp(X))

    def field(self, name: str) -> np.ndarray:
        out = np.zeros(self.N)
        lib().or_get_field(self.h, FIELDS[name], _dp(out))
        return out

    # equilibrium residual --------------------------------------------------
    def _res_state(self):
        X = [self.nodes(m) for m in range(len(self.nn))]
        X = np.concatenate(X) if X else np.zeros((0, 3))
        return self.t, self.field("phi"), self.field("psi"), X

    def residual(self) -> np.ndarray:
        """Convergence residual of an equilibrium run (the paper gives no
        criterion, Sec. 4; this is the reading used throughout): the largest
        change of phi and of psi over the cells and of any marker coordinate
        since the reference state (the previous call, or init), and the
        largest of the three divided by the steps in between.  The current
        state becomes the reference.  Returns [dphi, dpsi, dX, r]."""
        t0, phi0, psi0, X0 = self._res_ref
        t, phi, psi, X = cur = self._res_state()
        d = np.array([np.max(np.abs(phi - phi0)), np.max(np.abs(psi - psi0)),
                      np.max(np.abs(X - X0)) if X.size else 0.0])
        self._res_ref = cur
        r = d.max() / (t - t0) if t > t0 else 0.0
        return np.array([d[0], d[1], d[2], r])

    def masses(self) -> np.ndarray:
        out = np.zeros(3)
        lib().or_masses(self.h, _dp(out))
        return out

    # pieces used by the pins
    def mem_energy(self, m: int, which: int, X: np.ndarray) -> float:
        X = np.ascontiguousarray(X, dtype=np.float64)
        return lib().or_mem_energy(self.h, m, which, _dp(X))

    def mem_force(self, m: int, which: int, X: np.ndarray) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float64)
        F = np.zeros_like(X)
        lib().or_mem_force(self.h, m, which, _dp(X), _dp(F))
        return F

    def iprofile(self, Xall: np.ndarray):
        Xall = np.ascontiguousarray(Xall, dtype=np.float64)
        I = np.zeros(self.N)
        d = np.zeros(self.N)
        nb = lib().or_iprofile(self.h, _dp(Xall), _dp(I), _dp(d))
        return I, d, nb

    def coupling(self, psi: np.ndarray, Xall: np.ndarray, want_force=True):
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        Xall = np.ascontiguousarray(Xall, dtype=np.float64)
        F = np.zeros_like(Xall) if want_force else None
        E = lib().or_coupling(self.h, _dp(psi), _dp(Xall), _dp(F) if want_force else None)
        return E, F

    def potentials(self, rho, phi, psi, I):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, phi, psi, I)]
        out = [np.zeros(self.N) for _ in range(3)]
        lib().or_potentials(self.h, *[_dp(a) for a in arrs], *[_dp(o) for o in out])
        return out

    def spread(self, Xall, Fall):
        Xall = np.ascontiguousarray(Xall, dtype=np.float64)
        Fall = np.ascontiguousarray(Fall, dtype=np.float64)
        out = np.zeros(3 * self.N)
        lib().or_spread(self.h, _dp(Xall), _dp(Fall), _dp(out))
        return out.reshape(3, self.N)

    def grad_field(self, a):
        """Lattice gradient [3][N] of a scalar field (the step's stencil)."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        g = np.zeros(3 * self.N)
        lib().or_grad_field(self.h, _dp(a), _dp(g))
        return g.reshape(3, self.N)

    def lap_field(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        out = np.zeros(self.N)
        lib().or_lap_field(self.h, _dp(a), _dp(out))
        return out

    def force_fe(self, rho, phi, psi, I):
        """Free-energy force [3][N] of given fields as the step forms it."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, phi, psi, I)]
        F = np.zeros(3 * self.N)
        lib().or_force_fe(self.h, *[_dp(a) for a in arrs], _dp(F))
        return F.reshape(3, self.N)

    def bulk_pressure(self, rho, phi, psi):
        return lib().or_bulk_pressure(self.h, float(rho), float(phi), float(psi))

    def capsule_measures(self, m: int = 0, X=None):
        """(area, volume) of membrane m at X (default: current markers)."""
        X = self.nodes(m) if X is None else np.ascontiguousarray(X, dtype=np.float64)
        out = np.zeros(2)
        lib().or_capsule_measures(self.h, m, _dp(X), _dp(out))
        return out

    def contact_angle(self, m: int = 0, X=None, phi=None):
        """(mean, min, max) contact angle in degrees of membrane m with the
        phi = 0 interface, and the number of contact points."""
        X = self.nodes(m) if X is None else np.ascontiguousarray(X, dtype=np.float64)
        phi = self.field("phi") if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
        out = np.full(3, np.nan)
        n = lib().or_contact_angle(self.h, m, _dp(X), _dp(phi), _dp(out))
        return out, n

    def interp(self, X, field3):
        X = np.ascontiguousarray(X, dtype=np.float64)
        field3 = np.ascontiguousarray(field3, dtype=np.float64)
        U = np.zeros_like(X)
        lib().or_interp(self.h, X.shape[0], _dp(X), _dp(field3), _dp(U))
        return U


def round_to_format(x: float, fmt: str) -> float:
    """Round x to binary16 / bfloat16 / binary32 (ties to even)."""
    p, emin, maxv = {"f16": (11, -14, 65504.0), "bf16": (8, -126, 3.3895313892515355e38),
                     "f32": (24, -126, 3.4028234663852886e38)}[fmt]
    return lib().or_round(float(x), p, emin, maxv)


def peskin(r: float) -> float:
    return lib().or_peskin(float(r))
