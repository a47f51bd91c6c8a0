"""tlb_diagnostics_static, the diagnostics entry point that uses no device
memory from the caller (its reduction scratch is a fixed array inside the
library), must give the same results as tlb_diagnostics.  It is called twice
in a row, because every call reuses the same array.  This file is collected
last so that, if it fails, a run that stops at the first failure has already
run every other test."""
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


def _same(a, b):
    assert a.step == b.step and a.n_caps == b.n_caps
    # identical kernels in the same order: equal to rounding of the tree sums
    assert np.allclose(a.mass[:], b.mass[:], rtol=1e-14, atol=1e-12)
    assert np.allclose(a.area[:], b.area[:], rtol=1e-14, atol=1e-12)
    assert np.allclose(a.volume[:], b.volume[:], rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("which", ["3d_f32", "2d_f64"])
def test_static_diagnostics_match_the_arena_version(which):
    from paper_1906_03065_gb300 import Simulation
    wl = W.small_3d("f32") if which == "3d_f32" else W.capsule_2d("f64")
    g = Simulation(wl).init()
    first = g.diagnostics_static()
    _same(first, g.diagnostics())
    g.step(10)
    second = g.diagnostics_static()
    _same(second, g.diagnostics())
    assert second.step == 10
    assert abs(second.mass[0] - first.mass[0]) < 1e-6 * wl.params.ncells
