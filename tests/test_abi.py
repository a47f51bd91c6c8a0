"""The C-ABI library builds, loads and exports every symbol that
include/tlb.h declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tlb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tlb_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1906_03065_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "tlb_step" in names and "tlb_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_state_bytes_and_argument_errors_without_gpu():
    """tlb_state_bytes is host-only: sizes the arena, rejects bad arguments."""
    import paper_1906_03065_gb300 as T
    from paper_1906_03065_gb300 import build, workloads as W
    build.build()
    L = T.lib()
    wl = W.capsule_3d("f32")
    cp = T.make_params(wl.params)
    import numpy as np
    m = wl.membranes[0]
    X = np.ascontiguousarray(m.X)
    E = np.ascontiguousarray(m.elems, dtype=np.int32)
    mem = (T._Mem * 1)()
    mem[0].kind, mem[0].n_nodes, mem[0].n_elems = 1, X.shape[0], E.shape[0]
    mem[0].X0 = X.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    mem[0].elems = E.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    nb = ctypes.c_size_t(0)
    assert L.tlb_state_bytes(ctypes.byref(cp), mem, 1, ctypes.byref(nb)) == 0
    # two population buffers of 55 FP32 planes + 2 rest planes dominate
    N = 128 ** 3
    assert nb.value > 2 * 57 * N * 4
    assert nb.value < 4 * 57 * N * 4
    bad = T.make_params(wl.params)
    bad.tau = 0.4
    assert L.tlb_state_bytes(ctypes.byref(bad), mem, 1, ctypes.byref(nb)) == 1
    assert b"relaxation" in L.tlb_last_error()
    bad = T.make_params(wl.params)
    bad.dim = 4
    assert L.tlb_state_bytes(ctypes.byref(bad), mem, 1, ctypes.byref(nb)) == 1
