"""Checkpoint and resume (tlb_save / tlb_load) and the single-context run to
a residual tolerance (tlb_run) on the GPU."""
import numpy as np
import pytest

from paper_1906_03065_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_03065_gb300 import build
    build.build()


@pytest.mark.parametrize("which", ["3d_f32", "3d_f16", "2d_f64"])
def test_resume_is_bit_identical(which):
    """A context restored from a checkpoint taken after 7 steps, stepped 5
    more, equals the saved context stepped 5 more, bit for bit (populations,
    markers, the residual), though the restored one starts from the other
    population buffer and a fresh arena."""
    from paper_1906_03065_gb300 import Simulation
    wl = {"3d_f32": lambda: W.small_3d("f32"), "3d_f16": lambda: W.small_sweep_3d(1, seed=4, storage="f16")[0],
          "2d_f64": lambda: W.small_2d("f64")}[which]()
    a = Simulation(wl).init()
    a.step(7)
    a.residual()
    a.step(2)
    blob = a.save()
    a.step(5)
    ra = a.residual()
    b = Simulation(wl).load(blob)
    b.step(5)
    rb = b.residual()
    assert np.array_equal(a.pops(), b.pops())
    assert np.array_equal(a.nodes(0), b.nodes(0))
    assert np.array_equal(ra, rb)
    assert b.diagnostics().step == 14


def test_load_rejects_foreign_or_truncated_blobs():
    from paper_1906_03065_gb300 import Simulation, TLBError
    wl = W.small_3d("f32")
    a = Simulation(wl).init()
    blob = a.save()
    other = W.small_3d("f32")
    other.params.kappa1 = 0.02
    with pytest.raises(TLBError, match="other parameters"):
        Simulation(other).load(blob)
    with pytest.raises(TLBError, match="truncated"):
        Simulation(wl).load(blob[:-100])
    bad = blob.copy()
    bad[:8] = 0
    with pytest.raises(TLBError, match="not a checkpoint"):
        Simulation(wl).load(bad)


def test_run_stops_at_the_tolerance():
    """A state at rest converges at the first check; a capsule run goes on to
    max_steps with a residual above the tolerance."""
    from paper_1906_03065_gb300 import Simulation
    p = W.Params(dim=3, nx=26, ny=24, nz=20, wall_last=1, storage="f32", alpha=1.0, dc=8.0, interface_pos=-1.0)
    n = p.ncells
    rest = Simulation(W.Workload("rest", p, [])).init(
        Cf=np.stack([np.full(n, 0.55), np.full(n, 0.45), np.zeros(n)]), u=np.zeros((3, n)))
    t, r = rest.run(100, 10, 1e-6)
    assert t == 10 and r <= 1e-6
    cap = Simulation(W.small_3d("f32")).init()
    t, r = cap.run(40, 20, 1e-9)
    assert t == 40 and r > 1e-9
