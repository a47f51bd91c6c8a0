"""The paper's 2D validation experiments (Sec. 4.1) on the GPU, at half the
paper's size (R = 10 in a 120 x 60 periodic lattice) so that they run in
seconds:

* Galilean invariance: every fluid given a uniform U_x0 carries the capsule
  along at U_x0, and its shape, drift removed, is the stationary one;
* the symmetric case (kappa_1 = kappa_2) runs as the FP64 oracle does and
  stays mirror-symmetric about the interface up to the profile I's
  tie-break between equidistant mirror segments;
* softer capsules deform more at the same tensions, towards the pure liquid
  lens (reported beside them).
"""
import numpy as np
import pytest

from paper_1906_03065_gb300 import validation as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_03065_gb300 import build
    build.build()


R = 10.0
SYM = (8e-3, 8e-3, 5e-4)  # the highest tension ratio of the symmetric case


def _centred(X):
    return X[:, :2] - X[:, :2].mean(axis=0)


def test_galilean_invariance_of_the_capsule_shape():
    steps = 3000
    wls = [V.capsule_at_interface(SYM, 1e-3, 1e-2, U=U, R=R) for U in (0.0, 1e-3, 1e-2)]
    b = V.relax(wls, steps)
    X0 = b[0].nodes(0)
    for i, U in ((1, 1e-3), (2, 1e-2)):
        X = b[i].nodes(0)
        drift = (X[:, :2] - X0[:, :2]).mean(axis=0)
        # carried along at U (the capsule moves with the fluid)
        assert abs(drift[0] - U * steps) < 0.02 * U * steps + 0.05, (U, drift)
        dev = np.abs(_centred(X) - _centred(X0)).max()
        print(f"U = {U:g}: drift {drift}, shape deviation {dev:.3e}")
        assert dev < 0.05 * (U / 1e-2) + 0.005, (U, dev)
        assert abs(V.taylor_deformation(X) - V.taylor_deformation(X0)) < 2e-3


def test_symmetric_case_matches_the_oracle_and_stays_nearly_mirror_symmetric():
    """kappa_1 = kappa_2: the set-up is mirror-symmetric about the interface
    (C1 and C2 exchanged).  The discrete method keeps that symmetry only up
    to the nearest-element tie-break of the profile I (equidistant mirror
    segments go to the lower index), which the FP64 oracle shares: the GPU
    run equals the oracle's to 1e-9 lattice units, and both stay symmetric
    to a few hundredths of a lattice unit after 3000 steps."""
    import oracle
    oracle.build()
    oracle.set_threads(0)
    wl = V.capsule_at_interface(SYM, 1e-3, 1e-2, R=R)
    b = V.relax([wl], 3000)
    X = b[0].nodes(0)
    o = oracle.Oracle(wl, init=False)
    o.init(V.initial_fields(wl), None)
    o.step(3000)
    assert np.abs(X - o.nodes(0)).max() < 1e-9
    n = X.shape[0]
    yc = wl.params.ny / 2.0
    mirror = X[(n - np.arange(n)) % n]  # node k <-> node n - k (angles theta <-> -theta)
    assert np.abs(X[:, 0] - mirror[:, 0]).max() < 0.05
    assert np.abs((X[:, 1] - yc) + (mirror[:, 1] - yc)).max() < 0.05
    assert V.taylor_deformation(X) > 0.01  # the tensions have deformed it


def test_softer_capsules_deform_more():
    """At the same tensions the capsule deforms more the lower its modulus
    kappa_s (Sec. 4.1); the pure lens is reported beside them."""
    steps = 6000
    wls = [V.capsule_at_interface(SYM, ks, 1e-2, R=R) for ks in (1e-3, 1e-2, 1e-1)]
    b = V.relax(wls, steps)
    D = [V.taylor_deformation(b[i].nodes(0)) for i in range(3)]
    lens = V.capsule_at_interface(SYM, 0.0, 0.0, R=R, membrane=False)
    ring = V.capsule_at_interface(SYM, 1e-3, 1e-2, R=R)
    bl = V.relax([lens], steps, fields=[V.initial_fields(ring)])
    D_lens = V.lens_deformation(bl[0].field("psi"), (lens.params.ny, lens.params.nx))
    print(f"D for kappa_s 1e-3, 1e-2, 1e-1: {D}; lens (C3 field moments) {D_lens:.4f}")
    assert D[0] > D[1] > D[2] > 0.0


def test_capillary_bridge_matches_the_oracle():
    """Sec. 4.2 set-up (a C2 bridge between two capsules in C1) at half the
    paper's size, FP64: the GPU run equals the oracle's after 400 steps."""
    import oracle
    from paper_1906_03065_gb300 import Simulation
    oracle.build()
    oracle.set_threads(0)
    wl, rect = V.capillary_bridge(3e-3, 1e-2, R=R)
    C = V.initial_fields(wl, bridge=rect)
    g = Simulation(wl).init(C, None)
    o = oracle.Oracle(wl, init=False)
    o.init(C, None)
    g.step(400)
    o.step(400)
    for m in range(2):
        assert np.abs(g.nodes(m) - o.nodes(m)).max() < 1e-9
    for n in ("C1", "C2", "C3"):
        assert np.abs(g.field(n) - o.field(n)).max() < 1e-10, n


def test_bridge_deforms_softer_capsules_more():
    """Sec. 4.2 at the paper's size, gamma_12 / gamma_13 = 0.8 (kappa_1 =
    9e-3): the bridge compresses the capsules along the line joining them
    (L_c / H_c < 1), and a stiffer capsule ends shorter and wider than a soft
    one (larger L_c / H_c), as the paper reports; the two capsules, mirror
    images across the bridge, deform alike."""
    rows = V.bridge_sweep(kappa1_list=(9e-3,), ks_list=(1e-3, 1e-1), steps=20000, device="cuda:0")
    soft, stiff = rows[0]["aspect"], rows[1]["aspect"]
    print(f"L_c/H_c: ks 1e-3 {soft}, ks 1e-1 {stiff}")
    assert soft[0] < 1 and stiff[0] < 1
    assert stiff[0] > soft[0]
    for a in (soft, stiff):
        assert abs(a[0] - a[1]) < 0.02 * abs(a[0])


def test_deformation_sweep_batches_every_combination_as_if_alone():
    """The Sec. 4.1 sweep relaxes every (kappa, ks, kb) capsule in one batch;
    each lattice's result is the one it gets relaxed alone, bit for bit (the
    instances share kernels, not state)."""
    cases = [SYM, (8e-3, 8e-3, 4e-3)]
    rows = V.deformation_sweep(cases, ks_list=(1e-3, 1e-1), kb_list=(1e-2,), steps=500, lens=False)
    assert [(r["ks"], r["kappa"]) for r in rows] == [(ks, k) for ks in (1e-3, 1e-1) for k in cases]
    for r in rows:
        b = V.relax([V.capsule_at_interface(r["kappa"], r["ks"], r["kb"], storage="f32")], 500)
        assert V.taylor_deformation(b[0].nodes(0)) == r["D"]


def test_galilean_runs_report_drift_and_shape():
    """The Galilean rows carry the capsule along at U (drift close to U *
    steps) with the stationary shape (half the paper's size, 3000 steps)."""
    rows = V.galilean_runs(U_list=(1e-3, 1e-2), steps=3000, R=R)
    for r in rows:
        assert abs(r["drift"][0] - r["U_steps"]) < 0.02 * r["U_steps"] + 0.05, r
        assert r["shape_dev"] < 0.05 * (r["U"] / 1e-2) + 0.005, r
        assert abs(r["D"] - r["D_stationary"]) < 2e-3, r
