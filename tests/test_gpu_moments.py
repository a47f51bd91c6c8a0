"""Moment storage (TLB_STATE_MOMENTS): at tau = tau_phi = tau_psi = 1 with the
exact difference method every post-collision population is an equilibrium of
its cell (eq. LBE at tau = 1), so the library may keep 11 moments per cell
instead of the 3Q populations and rebuild each population in the pull.  It
is the same method executed another way, so it must match the FP64 oracle
as the population scheme does, and the population scheme itself up to
rounding."""
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


def _sim(wl):
    from paper_1906_03065_gb300 import Simulation
    return Simulation(wl)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _moments(wl):
    wl.params.state = "moments"
    return wl


def _fields(s):
    return {n: s.field(n) for n in ("C1", "C2", "C3")}


def test_capsule_2d_f64_2000_steps_matches_oracle():
    wl = _moments(W.capsule_2d("f64"))
    g, o = _sim(wl).init(), oracle.Oracle(wl)
    g.step(2000)
    o.step(2000)
    for n in ("C1", "C2", "C3"):
        assert np.abs(g.field(n) - o.field(n)).max() < 1e-10, n
    u = np.stack([o.field("ux"), o.field("uy")])
    assert np.abs(g.field("u")[:2] - u).max() < 1e-10
    assert np.abs(g.nodes(0) - o.nodes(0)).max() < 1e-10


def test_small_3d_f32_matches_oracle():
    """FP32 fields within 1e-4 (relative L-inf on C and u, lattice units on
    the markers) of the FP64 oracle, with walls, a ragged lattice and a
    capsule on the interface."""
    wl = _moments(W.small_3d("f32"))
    oracle.set_threads(0)
    g, o = _sim(wl).init(), oracle.Oracle(wl)
    g.step(300)
    o.step(300)
    for n in ("C1", "C2", "C3"):
        assert _rel(g.field(n), o.field(n)) < 1e-4, n
    uo = np.stack([o.field("ux"), o.field("uy"), o.field("uz")])
    assert _rel(g.field("u"), uo) < 1e-4
    assert np.abs(g.nodes(0) - o.nodes(0)).max() < 1e-4


def test_equals_the_population_scheme():
    """FP64: the moment-stored and the population-stored runs agree to
    rounding at every read-out (fields, populations, markers, FP64 totals,
    residual)."""
    a = _sim(W.capsule_2d("f64")).init()
    b = _sim(_moments(W.capsule_2d("f64"))).init()
    for n in (1, 37, 200):
        a.step(n)
        b.step(n)
        assert np.abs(a.pops() - b.pops()).max() < 1e-13, n
        assert np.abs(a.nodes(0) - b.nodes(0)).max() < 1e-12, n
        da, db = a.diagnostics(), b.diagnostics()
        assert np.allclose(da.mass[:], db.mass[:], rtol=0, atol=1e-10)
        ra, rb = a.residual(), b.residual()
        assert np.abs(ra - rb).max() < 1e-12


def test_checkpoint_continues_bit_for_bit():
    wl = _moments(W.small_3d("f32"))
    a = _sim(wl).init()
    a.step(25)
    blob = a.save()
    a.step(30)
    b = _sim(wl)
    b.load(blob)
    b.step(30)
    assert np.array_equal(a.pops(), b.pops())
    assert np.array_equal(a.nodes(0), b.nodes(0))


def test_written_populations_are_pulled():
    """Populations written by the caller are the state of the next step
    (they need not be equilibria): one step from a perturbed state matches
    the population scheme from the same state."""
    wl = W.small_2d("f64")
    o = oracle.Oracle(wl, init=False)
    C0, u0 = W.random_fields(wl.params, seed=4)
    o.init(C0, u0)
    rng = np.random.default_rng(5)
    c, w = o.lattice()
    P = o.pops() + 1e-3 * rng.standard_normal((3, o.Q, o.N)) * w[None, :, None]
    a = _sim(wl)
    a.init(C0, u0)
    a.set_pops(P)
    b = _sim(_moments(W.small_2d("f64")))
    b.init(C0, u0)
    b.set_pops(P)
    o.set_pops(P)
    for s in (a, b, o):
        s.step(3)
    assert np.abs(b.pops() - o.pops()).max() < 1e-12
    assert np.abs(b.pops() - a.pops()).max() < 1e-13


def test_refused_where_it_does_not_apply():
    from paper_1906_03065_gb300 import TLBError
    for tau, forcing, storage in ((0.8, "edm", "f64"), (1.0, "guo", "f64")):
        wl = _moments(W.small_2d(storage))
        wl.params.tau = wl.params.tau_phi = wl.params.tau_psi = tau
        wl.params.forcing = forcing
        with pytest.raises(TLBError):
            _sim(wl)
    with pytest.raises(TLBError):
        _sim(_moments(W.small_3d("f16")))
    g = _sim(_moments(W.small_2d("f64"))).init()
    with pytest.raises(TLBError):
        g.set_tile(1, 8)
    g.set_tile(16, 8)
    from paper_1906_03065_gb300 import Batch
    with pytest.raises(TLBError):
        Batch([_moments(W.small_2d("f64"))])


def test_pair_collide_stores_the_same_moments():
    """With moment storage the tau = 1 collide with two cells per thread
    (variants 22-27) writes the same 11 moments per cell as the single-cell
    collide."""
    wl = _moments(W.small_3d("f32"))
    a, b = _sim(wl).init(), _sim(wl).init()
    a.set_tile(14, 8)
    b.set_tile(23, 8)
    a.step(20)
    b.step(20)
    for n in ("C1", "C2", "C3", "u"):
        assert np.array_equal(a.field(n), b.field(n)), n
    assert np.array_equal(a.nodes(0), b.nodes(0))
