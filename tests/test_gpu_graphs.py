"""Step graphs: runs of 8 steps replayed from a captured CUDA graph launch the
same kernels on the same buffers as direct launches, so the state after any
mix of replays, direct steps, markers set from outside and a phase profile is
identical bit for bit to stepping with graphs off."""
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


def _cases():
    w3 = W.small_3d("f32")
    wm = W.small_3d("f32")
    wm.params.state = "moments"
    w16 = W.small_3d("f16", nx=36, ny=32, nz=30, radius=6.0, centre=(18.2, 16.1, 15.3))
    return [("2d_f64", W.small_2d("f64"), None), ("3d_f32", w3, None), ("3d_f32_general", W.small_3d("f32"), 6),
            ("3d_f32_moments", wm, None), ("3d_f16", w16, None)]


def _state(s):
    out = [s.field(n) for n in ("C1", "C2", "C3", "u")]
    out.append(s.nodes(0))
    return out


def _run(wl, variant, graphs):
    from paper_1906_03065_gb300 import Simulation
    s = Simulation(wl).init()
    if variant is not None:
        s.set_tile(variant, 4)
    s.set_graphs(graphs)
    s.step(3)
    s.step(21)          # two replays and five direct steps
    n21 = s.launches()
    X = s.nodes(0)
    X[:, 0] += 0.013     # markers set from outside: the next step runs direct
    s.set_nodes(0, X)
    s.step(17)
    s.profile(2)         # profiled steps run direct
    s.step(16)
    return _state(s), n21


@pytest.mark.parametrize("name,wl,variant", _cases(), ids=[c[0] for c in _cases()])
def test_graph_replay_is_bitwise_identical_to_direct_launches(name, wl, variant):
    a, na = _run(wl, variant, False)
    b, nb = _run(wl, variant, True)
    assert na == nb  # the replays count the kernels they hold
    for x, y in zip(a, b):
        assert np.array_equal(x, y), name


def test_graphs_follow_a_change_of_collide_variant():
    from paper_1906_03065_gb300 import Simulation
    wl = W.small_3d("f32")
    runs = []
    for graphs in (False, True):
        s = Simulation(wl).init()
        s.set_graphs(graphs)
        s.set_tile(13, 4)
        s.step(16)
        s.set_tile(14, 8)  # a graph captured with variant 13 must not replay
        s.step(16)
        runs.append(_state(s))
    for x, y in zip(*runs):
        assert np.array_equal(x, y)
