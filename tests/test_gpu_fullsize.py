"""Parity at the full workload sizes, in the launch configuration bench.py
times (autotuned collide), on outputs the FP64 oracle can compute: the
192x128x128 two-capsule bridge in FP16 storage, and two sampled instances of
the 64-instance FP16 sweep stepped as one batch."""
import numpy as np
import pytest

import oracle
from paper_1906_03065_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_03065_gb300 import build
    build.build()
    oracle.build()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _check(g, o, nmem, tc=2e-3, tu=5e-2, tx=1e-3):
    for n in ("C1", "C2", "C3"):
        assert _rel(g.field(n), o.field(n)) < tc, n
    uo = np.stack([o.field("ux"), o.field("uy"), o.field("uz")])
    assert _rel(g.field("u"), uo) < tu
    for m in range(nmem):
        assert np.abs(g.nodes(m) - o.nodes(m)).max() < tx, m


def test_bridge_3d_f16_full_size():
    from paper_1906_03065_gb300 import Simulation
    wl = W.bridge_3d("f16")
    g = Simulation(wl).init()
    g.autotune()
    o = oracle.Oracle(wl, emulate_storage=True)
    g.step(2)
    o.step(2)
    _check(g, o, 2)


def test_sweep_batch_full_size_sampled():
    from paper_1906_03065_gb300 import Batch
    wls = W.sweep_3d()
    b = Batch(wls).init()
    b.autotune()
    b.step(3)
    small = sorted(range(len(wls)), key=lambda i: wls[i].params.ncells)[:2]
    for i in small:
        o = oracle.Oracle(wls[i], emulate_storage=True)
        o.step(3)
        _check(b[i], o, 1)
