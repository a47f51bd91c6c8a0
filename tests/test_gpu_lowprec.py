"""FP16 / BF16 population storage (FP32 arithmetic): parity of the CUDA
path with the FP64 oracle that rounds its populations to the same storage
format after every step (f_i - w_i, g_i and h_i for i != 0 in the 16-bit
format; g_0, h_0 in binary32).

The two sides compute in FP32 and FP64, so a stored value that lies within
the FP32 rounding of a 16-bit midpoint can round differently: such events
move a population by one 16-bit unit (about 2^-11 or 2^-8 of its size).
The tolerances below bound the effect of those events over the run."""
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


# (storage, steps, tol on C1..C3, tol on u, tol on markers)
CASES = [("f16", 100, 2e-3, 5e-2, 1e-3), ("bf16", 100, 2e-2, 5e-1, 1e-2)]


@pytest.mark.parametrize("storage,steps,tc,tu,tx", CASES)
def test_low_precision_storage_matches_emulating_oracle(storage, steps, tc, tu, tx):
    from paper_1906_03065_gb300 import Simulation
    wl = W.small_3d(storage)
    g = Simulation(wl).init()
    o = oracle.Oracle(wl, emulate_storage=True)
    g.step(steps)
    o.step(steps)
    err = {n: _rel(g.field(n), o.field(n)) for n in ("C1", "C2", "C3")}
    ug = g.field("u")
    uo = np.stack([o.field("ux"), o.field("uy"), o.field("uz")])
    err["u"] = _rel(ug, uo)
    err["X"] = np.abs(g.nodes(0) - o.nodes(0)).max()
    print(storage, {k: f"{v:.2e}" for k, v in err.items()})
    for n in ("C1", "C2", "C3"):
        assert err[n] < tc, err
    assert err["u"] < tu, err
    assert err["X"] < tx, err
