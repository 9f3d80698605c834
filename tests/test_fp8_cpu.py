"""CPU pins of the FP8 input encoding shared by the oracle side of the FP8
parity tests: e4m3 rounding (OCP FP8 E4M3) and the per-side power-of-two
scale. The CUDA path implements its own conversion (cvt to e4m3 with
saturation); the GPU tests check that both give the same factors."""

import math

import numpy as np
import pytest

from synth import fp8_quantized, fp8_side_exponent, make_market, round_to_e4m3


def test_e4m3_rounding_matches_torch_cast():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 30, 100000), rng.normal(0, 0.01, 100000), rng.uniform(-448, 448, 50000),
                        np.ldexp(rng.integers(1, 16, 2000), -10) * rng.choice([-1, 1], 2000)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).double().numpy()
    np.testing.assert_array_equal(round_to_e4m3(x), ref)


def test_e4m3_format_values():
    # largest finite, saturation, smallest subnormal, ties to even, binade edges
    cases = {448.0: 448.0, 500.0: 448.0, 1e6: 448.0, -1e6: -448.0, 2.0 ** -9: 2.0 ** -9, 2.0 ** -10: 0.0,
             3 * 2.0 ** -10: 2 * 2.0 ** -9,  # 1.5 quanta -> 2 (even)
             1.0625: 1.0,  # halfway between 1 and 1.125 -> 1 (even mantissa)
             1.1875: 1.25,  # halfway between 1.125 and 1.25 -> 1.25 (even)
             240.0: 240.0, 248.0: 256.0, 2.0 ** -6: 2.0 ** -6, 0.0: 0.0}
    for x, want in cases.items():
        assert round_to_e4m3(np.float64(x)) == want, x
    # 8 values per binade: the e4m3 grid of [1, 2)
    grid = round_to_e4m3(np.linspace(1.0, 1.999, 1000))
    assert sorted(set(grid.tolist())) == [1 + i / 8 for i in range(8)] + [2.0]


def test_side_exponent_definition():
    rng = np.random.default_rng(1)
    for scale in (1e-3, 0.125, 1.0, 447.9, 448.0, 448.1, 3e4):
        A = (rng.normal(0, 1, (50, 7)) * scale).astype(np.float32)
        B = (rng.normal(0, 1, (50, 7)) * scale).astype(np.float32)
        k = fp8_side_exponent(A, B)
        mx = float(max(np.abs(A).max(), np.abs(B).max()))
        assert mx <= math.ldexp(448.0, k) and mx > math.ldexp(448.0, k - 1)
    assert fp8_side_exponent(np.zeros((2, 2)), np.zeros((2, 2))) == 0


def test_fp8_quantized_market():
    mk = make_market(300, 200, 24, sigma=0.5, seed=3, dtype="fp32")
    q, (kx, ky) = fp8_quantized(mk)
    for a, k in ((q.F, kx), (q.K, kx), (q.G, ky), (q.L, ky)):
        scaled = a.astype(np.float64) * 2.0 ** -k
        np.testing.assert_array_equal(round_to_e4m3(scaled), scaled)  # already on the e4m3 grid
    # half a quantum: at most 2^-4 relative for normal values, 2^(k-10) absolute below 2^(k-6)
    err = np.abs(q.F.astype(np.float64) - mk.F)
    bound = np.maximum(2.0 ** -4 * np.abs(mk.F.astype(np.float64)), 2.0 ** (kx - 10))
    assert np.all(err <= bound * (1 + 1e-12))
