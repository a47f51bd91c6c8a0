"""Batched sweep on the GPU: uneven instances stepped by the persistent,
graph-captured phase launches evolve exactly as when stepped alone, match
the FP64 oracle, report the oracle's residual, and retire when converged."""
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


def _pair(wls):
    from paper_1906_03065_gb300 import Batch, Simulation
    return Batch(wls).init(), [Simulation(wl).init() for wl in wls]


def test_batch_matches_single_instances_bitwise_f64():
    """Same kernel bodies, same arithmetic: in FP64 every instance's
    populations and markers equal those of the instance stepped alone, bit
    for bit, after an odd number of steps (graph launches plus one direct
    step) and after more steps on top; the launch count does not grow with
    the number of instances."""
    wls = [W.small_2d("f64"), W.small_2d("f64", nx=44, ny=40, centre=(21.1, 19.7)), W.small_2d("f64", nx=36)]
    b, alone = _pair(wls)
    for n, boxes in ((7, len(wls)), (6, 0)):
        b.step(n)
        # six phase launches per step (plus the marker boxes of freshly
        # initialised instances on the first call)
        assert b.launches() == 6 * n + boxes
        for s in alone:
            s.step(n)
        for i, s in enumerate(alone):
            Pb, Ps = b[i].pops(), s.pops()
            assert np.array_equal(Pb, Ps), (n, i, np.abs(Pb - Ps).max())
            assert np.array_equal(b[i].nodes(0), s.nodes(0)), (n, i, np.abs(b[i].nodes(0) - s.nodes(0)).max())


def test_batch_matches_single_instances_f32():
    """FP32 3D: the lattice update alone is bit-identical (no membrane); with
    membranes the FP32 membrane kernels, compiled into a different kernel,
    may contract multiply-adds differently, so instances agree to rounding:
    a few FP32 units of the populations and of the marker velocities."""
    p = W.Params(dim=3, nx=26, ny=24, nz=20, wall_last=1, storage="f32", alpha=1.0, dc=8.0, interface_pos=10.0)
    b, alone = _pair([W.Workload("nomem_26x24x20", p, [])])
    b.step(5)
    alone[0].step(5)
    assert np.array_equal(b[0].pops(), alone[0].pops())
    wls = W.small_sweep_3d(4, storage="f32")
    b, alone = _pair(wls)
    for n in (7, 6):
        b.step(n)
        for s in alone:
            s.step(n)
        for i, s in enumerate(alone):
            assert np.abs(b[i].pops() - s.pops()).max() < 1e-6, (n, i)
            assert np.abs(b[i].nodes(0) - s.nodes(0)).max() < 1e-8, (n, i)


def test_batch_f16_matches_emulating_oracle():
    """FP16 storage: each batched instance against the FP64 oracle that rounds
    its populations to binary16 after every step (the bounds of the
    single-lattice FP16 parity test)."""
    from paper_1906_03065_gb300 import Batch
    wls = W.small_sweep_3d(3, seed=11, storage="f16")
    b = Batch(wls).init()
    steps = 60
    b.step(steps)
    for i, wl in enumerate(wls):
        o = oracle.Oracle(wl, emulate_storage=True)
        o.step(steps)
        g = b[i]
        for n in ("C1", "C2", "C3"):
            assert _rel(g.field(n), o.field(n)) < 2e-3, (i, n)
        uo = np.stack([o.field("ux"), o.field("uy"), o.field("uz")])
        assert _rel(g.field("u"), uo) < 5e-2, i
        assert np.abs(g.nodes(0) - o.nodes(0)).max() < 1e-3, i


def test_residual_matches_oracle():
    """tlb_residual (single context) and the batched residual of tlb_batch_run
    against the oracle's residual after the same steps (FP32 storage: the
    changes are ~1e-3, FP32 rounding of the fields ~1e-7)."""
    from paper_1906_03065_gb300 import Batch, Simulation
    wl = W.small_3d("f32")
    g = Simulation(wl).init()
    o = oracle.Oracle(wl)
    for _ in range(2):
        g.step(10)
        o.step(10)
        rg, ro = g.residual(), o.residual()
        assert np.allclose(rg, ro, rtol=2e-3, atol=1e-7), (rg, ro)
    wls = W.small_sweep_3d(2, seed=3, storage="f32")
    b = Batch(wls).init()
    steps, res = b.run(max_steps=20, check_every=10, tol=0.0)
    assert list(steps) == [20, 20]
    for i, wl in enumerate(wls):
        o = oracle.Oracle(wl)
        o.step(10)
        o.residual()
        o.step(10)
        ro = o.residual()
        assert res[i] == pytest.approx(ro[3], rel=2e-3, abs=1e-8), (i, res[i], ro)


def test_batch_run_retires_converged_instances():
    """An instance at rest (uniform composition, no membrane) converges at the
    first check and stops; the capsule instance runs on to max_steps."""
    from paper_1906_03065_gb300 import Batch
    cap = W.small_sweep_3d(1, seed=5, storage="f32")[0]
    p = W.Params(dim=3, nx=26, ny=24, nz=20, wall_last=1, storage="f32", alpha=1.0, dc=8.0,
                 interface_pos=-1.0)
    rest = W.Workload("rest_26x24x20", p, [])
    b = Batch([rest, cap])
    n = p.ncells
    b[0].init(Cf=np.stack([np.full(n, 0.55), np.full(n, 0.45), np.zeros(n)]), u=np.zeros((3, n)))
    b[1].init()
    before = b[0].pops()
    # FP32 populations of a state at rest settle by rounding (~1e-8 per step)
    steps, res = b.run(max_steps=40, check_every=10, tol=1e-6)
    assert list(steps) == [10, 40], res
    assert res[0] <= 1e-6 and res[1] > 1e-5, res
    after = b[0].pops()
    assert np.abs(after - before).max() < 1e-6
    # a retired instance is left alone by further batched steps
    b.step(4)
    assert np.array_equal(b[0].pops(), after)
    b.set_active([1, 1])
    b.step(2)
    assert b.launches() == 12
