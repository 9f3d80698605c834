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


def test_serving_stream_replays_across_rates():
    """Every offered rate replays the same requests: a stream's first requests
    do not depend on its length, and arrivals scale as 1 / rate."""
    from synth import serving_workload
    long = serving_workload(12, rate=1.0, lo=100, hi=400, seed=5)
    short = serving_workload(8, rate=40.0, lo=100, hi=400, seed=5)
    for a, b in zip(long, short):
        assert a["key"] == b["key"] and a["resolve"] == b["resolve"]
        for name in ("F", "K", "G", "L", "n", "m"):
            assert np.array_equal(a[name], b[name])
        assert abs(a["t"] / 40.0 - b["t"]) <= 1e-12 * max(1.0, b["t"])
    t = np.array([w["t"] for w in long])
    assert np.all(np.diff(t) > 0)
    # re-solves repeat an earlier market (same key, same shape, perturbed bf16 factors)
    assert sum(w["resolve"] for w in long) >= 2
    first = {}
    for w in long:
        if w["resolve"]:
            base = first[w["key"]]
            assert base["F"].shape == w["F"].shape and not np.array_equal(base["F"], w["F"])
            assert np.array_equal(round_to_bf16(w["F"]), w["F"])
        else:
            first[w["key"]] = w
