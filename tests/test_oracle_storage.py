"""Pins of the oracle's storage rounding (bf16 / fp16, round to nearest, ties
to even) against PyTorch's CPU conversions and hand-picked ties."""
import numpy as np
import pytest
import torch

import oracle


@pytest.mark.parametrize("fmt,dt", [("bf16", torch.bfloat16), ("f16", torch.float16)])
def test_rounding_matches_the_library_conversion(fmt, dt):
    rng = np.random.default_rng(0)
    x = (rng.normal(size=200_000) * 10.0 ** rng.uniform(-9, 6, 200_000)).astype(np.float32)
    got = oracle.round_storage(x.astype(np.float64), fmt)
    ref = torch.from_numpy(x).to(dt).double().numpy()
    np.testing.assert_array_equal(got, ref)


def test_ties_go_to_even_and_range_limits():
    r = oracle.round_storage
    # bf16 keeps 8 significant bits: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert r(1 + 2.0 ** -8, "bf16") == 1.0
    assert r(1 + 3 * 2.0 ** -8, "bf16") == 1 + 2 * 2.0 ** -7
    assert r(1 + 2.0 ** -11, "f16") == 1.0
    assert r(1 + 3 * 2.0 ** -11, "f16") == 1 + 2 * 2.0 ** -10
    # fp16: subnormal quantum 2^-24 below 2^-14; 65504 is the largest finite value
    assert r(1.5 * 2.0 ** -24, "f16") == 2 * 2.0 ** -24
    assert r(2.5 * 2.0 ** -24, "f16") == 2 * 2.0 ** -24
    assert r(65519.0, "f16") == 65504.0 and np.isinf(r(65520.0, "f16"))
    assert r(-3.0, "bf16") == -3.0 and r(0.0, "f16") == 0.0
