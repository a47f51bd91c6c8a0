"""Pin of the oracle's storage-rounding emulation (used for the FP16 / BF16
population storage parity): it must reproduce IEEE round-to-nearest-even
into binary16, bfloat16 and binary32 exactly, including ties, subnormals and
overflow, which numpy and torch implement (no GPU)."""
import numpy as np
import pytest

import oracle


def _torch_bf16(x):
    torch = pytest.importorskip("torch")
    return torch.tensor(x, dtype=torch.float64).to(torch.float32).to(torch.bfloat16).double().numpy()


def test_random_values_match_library_rounding():
    rng = np.random.default_rng(0)
    xs = rng.normal(size=3000) * np.logspace(-9, 4, 3000)
    r16 = np.array([oracle.round_to_format(x, "f16") for x in xs])
    assert np.array_equal(r16, xs.astype(np.float16).astype(np.float64))
    r32 = np.array([oracle.round_to_format(x, "f32") for x in xs])
    assert np.array_equal(r32, xs.astype(np.float32).astype(np.float64))
    # bfloat16 via float32 is exact when x is already a float32 (no double rounding)
    x32 = xs.astype(np.float32).astype(np.float64)
    rb = np.array([oracle.round_to_format(x, "bf16") for x in x32])
    assert np.array_equal(rb, _torch_bf16(x32))


def test_ties_subnormals_and_overflow():
    h = 2.0 ** -11  # half the spacing of binary16 at 1
    assert oracle.round_to_format(1 + h, "f16") == 1.0             # tie -> even
    assert oracle.round_to_format(1 + 3 * h, "f16") == 1 + 4 * h   # tie -> even (up)
    assert oracle.round_to_format(2.0 ** -24, "f16") == 2.0 ** -24  # smallest subnormal
    assert oracle.round_to_format(2.0 ** -26, "f16") == 0.0        # below half of it
    assert oracle.round_to_format(3 * 2.0 ** -26, "f16") == 2.0 ** -24
    assert oracle.round_to_format(65504.0, "f16") == 65504.0
    assert oracle.round_to_format(70000.0, "f16") == np.inf
    b = 2.0 ** -8
    assert oracle.round_to_format(1 + b, "bf16") == 1.0
    assert oracle.round_to_format(1 + 3 * b, "bf16") == 1 + 4 * b
