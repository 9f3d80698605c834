"""CPU pins of the FP8 input encoding shared by the oracle side of the FP8
parity tests: e4m3 rounding (OCP FP8 E4M3), its bit patterns, and the
per-row power-of-two scales. The CUDA path implements its own conversion (cvt
to e4m3 with saturation) and its own choice of the scales; the GPU tests check
that both give the same factors."""

import math

import numpy as np
import pytest

from synth import e4m3_bits, fp8_encoded, fp8_exponent, fp8_quantized, fp8_row_exponents, make_market, round_to_e4m3


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


def test_exponent_definition():
    rng = np.random.default_rng(1)
    for scale in (1e-3, 0.125, 1.0, 447.9, 448.0, 448.1, 3e4):
        A = (rng.normal(0, 1, (50, 7)) * scale).astype(np.float32)
        B = (rng.normal(0, 1, (50, 7)) * scale).astype(np.float32)
        k = fp8_row_exponents(A, B)
        mx = np.maximum(np.abs(A).max(axis=1), np.abs(B).max(axis=1)).astype(np.float64)
        assert np.all(mx <= np.ldexp(448.0, k)) and np.all(mx > np.ldexp(448.0, k - 1))
    # exact edges: 448 * 2^k itself belongs to k, the next float above to k + 1
    for k in (-20, -1, 0, 3):
        edge = math.ldexp(448.0, k)
        assert fp8_exponent(edge) == k and fp8_exponent(np.nextafter(edge, np.inf)) == k + 1
    assert fp8_exponent(0.0) == 0
    assert np.all(fp8_row_exponents(np.zeros((2, 2)), np.zeros((2, 2))) == 0)


def test_e4m3_bits_match_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    rng = np.random.default_rng(4)
    x = round_to_e4m3(np.concatenate([rng.normal(0, 30, 20000), rng.normal(0, 0.01, 20000),
                                      np.ldexp(rng.integers(0, 8, 500), -9), [0.0, -0.0, 448.0, -448.0]]))
    want = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(e4m3_bits(x), want)


def test_fp8_quantized_market():
    mk = make_market(300, 200, 24, sigma=0.5, seed=3, dtype="fp32")
    q, (kx, ky) = fp8_quantized(mk)
    for a, k in ((q.F, kx), (q.K, kx), (q.G, ky), (q.L, ky)):
        scaled = a.astype(np.float64) / np.ldexp(1.0, k)[:, None]
        np.testing.assert_array_equal(round_to_e4m3(scaled), scaled)  # already on the e4m3 grid
        assert np.all(np.abs(scaled).max(axis=1) <= 448.0)
    # half a quantum: at most 2^-4 relative for normal values, 2^(k_r-10) absolute below 2^(k_r-6)
    err = np.abs(q.F.astype(np.float64) - mk.F)
    bound = np.maximum(2.0 ** -4 * np.abs(mk.F.astype(np.float64)), np.ldexp(1.0, kx - 10)[:, None])
    assert np.all(err <= bound * (1 + 1e-12))
    # the caller's encoding: bytes and scales decode to the same factors
    F8, K8, G8, L8, sx, sy = fp8_encoded(mk)
    torch = pytest.importorskip("torch")
    if hasattr(torch, "float8_e4m3fn"):
        dec = lambda b, s: torch.from_numpy(b).view(torch.float8_e4m3fn).double().numpy() * s.astype(np.float64)[:, None]
        np.testing.assert_array_equal(dec(F8, sx), q.F)
        np.testing.assert_array_equal(dec(L8, sy), q.L)


def test_row_scales_keep_small_rows_precise():
    """Rows whose entries are 30,000 times smaller than the side's largest
    keep the relative precision of e4m3 (3 mantissa bits) with per-row scales;
    one scale per side pushes them into the subnormal range (quantum 2^-9 of
    the side's scale)."""
    rng = np.random.default_rng(6)
    A = rng.normal(0, 1, (64, 32))
    B = rng.normal(0, 1, (64, 32))
    A[::2] *= 3e-5  # the whole row [F_r | K_r] is small
    B[::2] *= 3e-5
    mk = make_market(64, 8, 32, sigma=0.5, seed=1, dtype="fp32")
    mk = mk.__class__(**{**mk.__dict__, "F": A.astype(np.float32), "K": B.astype(np.float32)})
    q, _ = fp8_quantized(mk)
    small = np.abs(q.F[::2].astype(np.float64) - mk.F[::2]) / np.abs(mk.F[::2].astype(np.float64))
    assert np.median(small) < 2.0 ** -5
    k_side = fp8_exponent(max(np.abs(A).max(), np.abs(B).max()))
    per_side = np.abs(round_to_e4m3(A[::2] / 2.0 ** k_side) * 2.0 ** k_side - A[::2]) / np.abs(A[::2])
    assert np.median(per_side) > 4 * np.median(small)
