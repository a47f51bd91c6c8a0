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


def _inst_descs(wls, keep):
    import paper_1906_03065_gb300 as T
    descs = (T._Inst * len(wls))()
    for i, wl in enumerate(wls):
        descs[i].params = T.make_params(wl.params)
        mems = T._marshal_membranes(wl, keep)
        keep.append(mems)
        descs[i].mems = ctypes.cast(mems, ctypes.POINTER(T._Mem))
        descs[i].n_mem = len(wl.membranes)
    return descs


def test_batch_state_bytes_without_gpu():
    """The batch arena is the instances' arenas (256-byte aligned) plus a few
    KB of tables per instance; mixed dim/storage and empty batches are
    rejected (host-only calls)."""
    import paper_1906_03065_gb300 as T
    from paper_1906_03065_gb300 import build, workloads as W
    build.build()
    L = T.lib()
    keep = []
    wls = W.small_sweep_3d(3, storage="f16")
    descs = _inst_descs(wls, keep)
    total = ctypes.c_size_t(0)
    assert L.tlb_batch_state_bytes(descs, 3, ctypes.byref(total)) == 0
    single = 0
    for i in range(3):
        nb = ctypes.c_size_t(0)
        assert L.tlb_state_bytes(ctypes.byref(descs[i].params), descs[i].mems, 1, ctypes.byref(nb)) == 0
        single += (nb.value + 255) // 256 * 256
    assert single < total.value < single + 3 * 8192
    assert L.tlb_batch_state_bytes(descs, 0, ctypes.byref(total)) == 1
    mixed = _inst_descs(W.small_sweep_3d(2, storage="f16") + W.small_sweep_3d(1, storage="f32"), keep)
    assert L.tlb_batch_state_bytes(mixed, 3, ctypes.byref(total)) == 1
    assert b"same dim and storage" in L.tlb_last_error()
    bad = _inst_descs(W.small_sweep_3d(2, storage="f16"), keep)
    bad[1].params.tau = 0.3
    assert L.tlb_batch_state_bytes(bad, 2, ctypes.byref(total)) == 1
    assert b"batch instance 1" in L.tlb_last_error()
