"""The seeded generators: determinism, shapes, and bf16 rounding."""

import numpy as np
import torch

from synth import bf16_bits, dense_job_market, make_market, round_to_bf16


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=10000).astype(np.float32),
                        np.array([1.0, -2.5, 3.0e-30, 1.00390625, 1.01171875], np.float32)])
    ours = round_to_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(ours, ref)
    bits = bf16_bits(ours)
    np.testing.assert_array_equal(bits, torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16))


def test_generators_are_seeded():
    a = make_market(50, 70, 8, sigma=0.5, seed=3, bias_x=True, bias_y=True, n_kind="uniform1to3")
    b = make_market(50, 70, 8, sigma=0.5, seed=3, bias_x=True, bias_y=True, n_kind="uniform1to3")
    for k in ("F", "K", "G", "L", "bias_x", "bias_y", "n", "m"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert a.F.shape == (50, 8) and a.G.shape == (70, 8)
    assert set(np.unique(a.n)) <= {1.0, 2.0, 3.0}
    np.testing.assert_array_equal(round_to_bf16(a.F), a.F)


def test_job_market_recipe():
    mk = dense_job_market(N=200, M=100)
    assert mk.bias_x is None and mk.bias_y is not None and np.all(mk.bias_y > 0)
    assert set(np.unique(mk.m)) <= {1.0, 2.0, 3.0, 4.0, 5.0}
    assert np.all(mk.n == 1.0) and mk.sigma == 0.5 and mk.dtype == "fp32"
