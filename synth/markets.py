"""Seeded generators for synthetic matching markets.

Every workload of the benchmark and of the tests comes from here. A market is
the input of the matrix-factorisation IPFP: factor matrices F, K (candidates,
N x d) and G, L (employers, M x d), optional additive popularity biases per
user, capacities n (N) and m (M), and the entropy scale sigma (= beta).

Values are drawn with numpy's PCG64 generator from a fixed seed, in float32,
then rounded (round-to-nearest-even) to the element type the device computes
in. The arrays stored in a :class:`Market` are exactly the values the device
sees, so a float64 computation on them measures the kernel and not the
quantisation.

Recipes (shapes and distributions follow the paper's Sec. 4.2 benchmark,
factors U[0, 1/sqrt(D)] with equal capacities, and the larger job-market
shapes of the benchmark configurations):

* ``plain_dense_market``: N = M = 1000, d = 16, factors N(0, 1/d), n = m = 1,
  sigma = 1.
* ``dense_job_market``: N = 20000 candidates, M = 10000 jobs, d = 32, factors
  N(0, 1/d), a LogNormal(0, 1) popularity bias on jobs, n = 1, job capacities
  uniform on {1..5}, sigma = 0.5, float32.
* ``fused_market``: N = M = 1e6, d = 64, bf16 factors N(0, 1/d), LogNormal(0, 1)
  popularity biases on both sides (float32), n = m = 1, sigma = 0.5.
* ``paper_shaped_market``: N = M, D = 50, factors U[0, 1/sqrt(D)],
  n = m = 1 (C = N), sigma = 1.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even).

    Returns float32 values that are exactly representable in bfloat16.
    """
    a = np.ascontiguousarray(x, dtype=np.float32)
    bits = a.view(np.uint32)
    # finite inputs: bits + bias <= 0xFF7FFFFF + 0x8000 stays below 2^32
    bias = ((bits >> np.uint32(16)) & np.uint32(1)) + np.uint32(0x7FFF)
    out = (bits + bias) & np.uint32(0xFFFF0000)
    return out.view(np.float32).reshape(a.shape)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """The bfloat16 bit patterns (uint16) of float32 values that are already
    bfloat16-representable (output of :func:`round_to_bf16`)."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    bits = a.view(np.uint32)
    if np.any(bits & np.uint32(0xFFFF)):
        raise ValueError("values are not bfloat16-representable; call round_to_bf16 first")
    return (bits >> np.uint32(16)).astype(np.uint16).reshape(a.shape)


@dataclasses.dataclass
class Market:
    """One synthetic market, values as the device sees them."""

    F: np.ndarray  # (N, d) float32
    K: np.ndarray  # (N, d) float32
    G: np.ndarray  # (M, d) float32
    L: np.ndarray  # (M, d) float32
    bias_x: Optional[np.ndarray]  # (N,) float32 or None
    bias_y: Optional[np.ndarray]  # (M,) float32 or None
    n: np.ndarray  # (N,) float64 capacities of side X
    m: np.ndarray  # (M,) float64 capacities of side Y
    sigma: float
    dtype: str  # "bf16" or "fp32": element type of F, K, G, L on the device
    seed: int
    recipe: str

    @property
    def N(self) -> int:
        return int(self.F.shape[0])

    @property
    def M(self) -> int:
        return int(self.G.shape[0])

    @property
    def d(self) -> int:
        return int(self.F.shape[1])

    def f64(self) -> dict:
        """float64 copies of every array (what the oracle consumes)."""
        out = {k: getattr(self, k).astype(np.float64) for k in ("F", "K", "G", "L", "n", "m")}
        out["bias_x"] = None if self.bias_x is None else self.bias_x.astype(np.float64)
        out["bias_y"] = None if self.bias_y is None else self.bias_y.astype(np.float64)
        out["sigma"] = float(self.sigma)
        return out

    def swapped(self) -> "Market":
        """The same market with the two sides exchanged (X <-> Y)."""
        return dataclasses.replace(
            self, F=self.G, K=self.L, G=self.F, L=self.K,
            bias_x=self.bias_y, bias_y=self.bias_x, n=self.m, m=self.n,
            recipe=self.recipe + "/swapped")


def _capacities(rng: np.random.Generator, size: int, kind: str) -> np.ndarray:
    if kind == "unit":
        return np.ones(size, dtype=np.float64)
    if kind == "uniform1to5":
        return rng.integers(1, 6, size=size).astype(np.float64)
    if kind == "uniform1to3":
        return rng.integers(1, 4, size=size).astype(np.float64)
    if kind == "uniform_real":
        return rng.uniform(0.5, 2.0, size=size)
    raise ValueError(f"unknown capacity kind {kind!r}")


def _factors(rng: np.random.Generator, rows: int, d: int, dist: str) -> np.ndarray:
    if dist == "normal":
        return rng.standard_normal((rows, d), dtype=np.float32) * np.float32(1.0 / math.sqrt(d))
    if dist == "uniform":
        return rng.random((rows, d), dtype=np.float32) * np.float32(1.0 / math.sqrt(d))
    raise ValueError(f"unknown factor distribution {dist!r}")


E4M3_MAX = 448.0


def round_to_e4m3(x) -> np.ndarray:
    """Nearest OCP FP8 E4M3 value (4 exponent bits with bias 7, 3 mantissa
    bits, subnormal quantum 2^-9, no infinities, largest finite 448), ties to
    even, saturating at +-448. Returns float64 (every e4m3 value is exact)."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, ex = np.frexp(a)              # a = m * 2^ex with m in [0.5, 1)
    e = np.maximum(ex - 1, -6)       # binade; below 2^-6 the quantum stays 2^-9
    q = np.ldexp(1.0, e - 3)
    r = np.minimum(np.round(a / q) * q, E4M3_MAX)
    return np.copysign(r, x)


def fp8_exponent(mx) -> np.ndarray:
    """Smallest integer k with mx <= 448 * 2^k, elementwise (0 where mx is 0)."""
    mx = np.asarray(mx, np.float64)
    k = np.frexp(np.where(mx > 0.0, mx / E4M3_MAX, 1.0))[1].astype(np.int64)
    k = np.where(np.ldexp(E4M3_MAX, k - 1) >= mx, k - 1, k)
    k = np.where(np.ldexp(E4M3_MAX, k) < mx, k + 1, k)
    return np.where(mx > 0.0, k, 0)


def fp8_row_exponents(A, B) -> np.ndarray:
    """Per row r of [A | B]: the smallest integer k_r with max_i |entry| <= 448 * 2^k_r."""
    mx = np.maximum(np.max(np.abs(np.asarray(A, np.float64)), axis=1), np.max(np.abs(np.asarray(B, np.float64)), axis=1))
    return fp8_exponent(mx)


def fp8_quantized(mk: "Market", per: str = "row"):
    """The factors an FP8 market computes with: row r of [F | K] (resp. of
    [G | L]) scaled by 2^-k_r (fp8_row_exponents; per="side": every row by the
    side's exponent, that of the side's largest |entry|), rounded to e4m3 and
    scaled back; exact in float32. Returns (market, (k_X, k_Y)) with the
    per-row exponents."""
    kx = fp8_row_exponents(mk.F, mk.K)
    ky = fp8_row_exponents(mk.G, mk.L)
    if per == "side":
        kx = np.full_like(kx, fp8_exponent(max(np.abs(mk.F).max(), np.abs(mk.K).max())))
        ky = np.full_like(ky, fp8_exponent(max(np.abs(mk.G).max(), np.abs(mk.L).max())))

    def q(a, k):
        sc = np.ldexp(1.0, k)[:, None]
        return (round_to_e4m3(np.asarray(a, np.float64) / sc) * sc).astype(np.float32)

    return dataclasses.replace(mk, F=q(mk.F, kx), K=q(mk.K, kx), G=q(mk.G, ky), L=q(mk.L, ky), dtype="fp8"), (kx, ky)


def e4m3_bits(x) -> np.ndarray:
    """Bit patterns (uint8) of e4m3 values x (already on the e4m3 grid):
    sign, 4 exponent bits with bias 7, 3 mantissa bits; exponent field 0 holds
    the subnormals, multiples of 2^-9."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    sub = a < 2.0 ** -6
    _, ex = np.frexp(np.where(sub, 1.0, a))
    e = ex - 1
    field = np.where(sub, 0, e + 7)
    mant = np.where(sub, a / 2.0 ** -9, (np.where(sub, 1.0, a) / np.ldexp(1.0, e) - 1.0) * 8.0)
    bits = (np.signbit(x).astype(np.int64) << 7) | (field.astype(np.int64) << 3) | np.rint(mant).astype(np.int64)
    return bits.astype(np.uint8)


def fp8_encoded(mk: "Market"):
    """The same quantization as fp8_quantized as a caller would hand it over:
    e4m3 bytes of F, K, G, L (uint8) and per-row FP32 scales 2^k."""
    kx = fp8_row_exponents(mk.F, mk.K)
    ky = fp8_row_exponents(mk.G, mk.L)

    def enc(a, k):
        return e4m3_bits(round_to_e4m3(np.asarray(a, np.float64) / np.ldexp(1.0, k)[:, None]))

    return (enc(mk.F, kx), enc(mk.K, kx), enc(mk.G, ky), enc(mk.L, ky),
            np.ldexp(1.0, kx).astype(np.float32), np.ldexp(1.0, ky).astype(np.float32))


def make_market(N: int, M: int, d: int, *, sigma: float, seed: int,
                dist: str = "normal", bias_x: bool = False, bias_y: bool = False,
                n_kind: str = "unit", m_kind: str = "unit", dtype: str = "bf16",
                factor_scale: float = 1.0, recipe: str = "custom") -> Market:
    """Draw one market. Draw order (fixed): F, K, G, L, bias_x, bias_y, n, m."""
    if dtype not in ("bf16", "fp32"):
        raise ValueError("dtype must be 'bf16' or 'fp32'")
    rng = np.random.default_rng(seed)
    mats = []
    for rows in (N, N, M, M):
        a = _factors(rng, rows, d, dist)
        if factor_scale != 1.0:
            a = a * np.float32(factor_scale)
        mats.append(round_to_bf16(a) if dtype == "bf16" else a.astype(np.float32))
    F, K, G, L = mats
    bx = rng.lognormal(0.0, 1.0, size=N).astype(np.float32) if bias_x else None
    by = rng.lognormal(0.0, 1.0, size=M).astype(np.float32) if bias_y else None
    n = _capacities(rng, N, n_kind)
    m = _capacities(rng, M, m_kind)
    return Market(F, K, G, L, bx, by, n, m, float(sigma), dtype, seed, recipe)


def plain_dense_market(N: int = 1000, M: int = 1000, d: int = 16, seed: int = 1000,
                       dtype: str = "fp32") -> Market:
    """Balanced plain market: factors N(0, 1/d), unit capacities, sigma = 1."""
    return make_market(N, M, d, sigma=1.0, seed=seed, dtype=dtype,
                       recipe=f"plain N={N} M={M} d={d}")


def dense_job_market(N: int = 20000, M: int = 10000, d: int = 32, seed: int = 1001,
                     dtype: str = "fp32") -> Market:
    """Job market for the materialised-kernel path: lognormal job popularity,
    job capacities uniform on {1..5}, sigma = 0.5."""
    return make_market(N, M, d, sigma=0.5, seed=seed, bias_y=True, m_kind="uniform1to5",
                       dtype=dtype, recipe=f"job N={N} M={M} d={d}")


def fused_market(N: int = 1_000_000, M: int = 1_000_000, d: int = 64, seed: int = 1002,
                 dtype: str = "bf16", sigma: float = 0.5) -> Market:
    """Large balanced market for the on-the-fly path: bf16 factors N(0, 1/d),
    lognormal popularity biases on both sides, unit capacities, sigma = 0.5
    (another sigma for profiling cases of other exponent ranges)."""
    return make_market(N, M, d, sigma=sigma, seed=seed, bias_x=True, bias_y=True,
                       dtype=dtype, recipe=f"fused N={N} M={M} d={d}" + ("" if sigma == 0.5 else f" sigma={sigma}"))


def paper_shaped_market(N: int, D: int = 50, seed: int = 1005, dtype: str = "bf16") -> Market:
    """Sec. 4.2 shape: N = M, factors U[0, 1/sqrt(D)], n = m = C/N with C = N, beta = 1."""
    return make_market(N, N, D, sigma=1.0, seed=seed, dist="uniform", dtype=dtype,
                       recipe=f"paper N={N} D={D}")


def batched_market_sizes(count: int = 512, lo: int = 100, hi: int = 50_000,
                         seed: int = 1003) -> list:
    """(N, M, capacity kind) of many independent markets; sizes log-uniform."""
    rng = np.random.default_rng(seed)
    ln = rng.uniform(math.log(lo), math.log(hi), size=(count, 2))
    sizes = np.rint(np.exp(ln)).astype(np.int64)
    kinds = ["unit" if i % 2 == 0 else "uniform1to3" for i in range(count)]
    return [(int(a), int(b), k) for (a, b), k in zip(sizes, kinds)]


def batched_markets(count: int = 512, lo: int = 100, hi: int = 50_000, d: int = 32, sigma: float = 1.0,
                    seed: int = 1003) -> list:
    """The independent markets of the batched workload: per-side sizes from
    batched_market_sizes (log-uniform in [lo, hi]); bf16 factors N(0, 1/d)
    sliced at seeded offsets from one seeded pool per matrix (so 512 markets
    are drawn in a second); capacities unit on both sides for even-indexed
    markets and uniform on {1..3} per user for odd ones; no biases."""
    sizes = batched_market_sizes(count, lo, hi, seed)
    rng = np.random.default_rng(seed + 1)
    pools = [round_to_bf16(_factors(rng, hi, d, "normal")) for _ in range(4)]
    out = []
    for i, (N, M, kind) in enumerate(sizes):
        mats = []
        for pool, rows in zip(pools, (N, N, M, M)):
            off = int(rng.integers(0, hi - rows + 1))
            mats.append(np.ascontiguousarray(pool[off:off + rows]))
        n = _capacities(rng, N, kind)
        m = _capacities(rng, M, kind)
        out.append(Market(mats[0], mats[1], mats[2], mats[3], None, None, n, m, float(sigma), "bf16",
                          seed * 100000 + i, f"batched #{i} N={N} M={M} d={d} {kind}"))
    return out


def serving_workload(count: int, rate: float = 200.0, lo: int = 1000, hi: int = 200_000, resolve_frac: float = 0.3,
                     perturb_std: float = 0.01, sigma: float = 1.0, seed: int = 1004, dims=(32, 64)) -> list:
    """A Poisson stream of solve requests: arrival times (rate per second),
    per-side sizes log-uniform in [lo, hi], d drawn from `dims`, bf16 factors
    N(0, 1/d) sliced from a seeded pool, capacities uniform on {1..3}, and a
    fraction of re-solves that repeat an earlier request's market with its
    factors perturbed by N(0, perturb_std^2) (same key, so a server can warm
    start). Returns a list of dicts with rid, t, key, F, K, G, L, n, m, sigma.

    The arrival times come from a generator of their own: the first requests
    of a stream are the same for every count and rate, and at rate r their
    arrivals are the rate-1 arrivals divided by r."""
    rng = np.random.default_rng(seed)
    pools = {}
    for d in dims:
        prng = np.random.default_rng(seed + 17 * d)
        pools[d] = [round_to_bf16(_factors(prng, hi, d, "normal")) for _ in range(4)]
    t = np.cumsum(np.random.default_rng([seed, 1]).exponential(1.0, size=count)) / rate
    out = []
    for i in range(count):
        if out and rng.random() < resolve_frac:
            base = out[int(rng.integers(0, len(out)))]
            d = base["F"].shape[1]
            mats = [round_to_bf16(a + rng.standard_normal(a.shape, dtype=np.float32) * np.float32(perturb_std))
                    for a in (base["F"], base["K"], base["G"], base["L"])]
            out.append(dict(rid=i, t=float(t[i]), key=base["key"], F=mats[0], K=mats[1], G=mats[2], L=mats[3],
                            n=base["n"], m=base["m"], sigma=sigma, resolve=True))
            continue
        N, M = (int(v) for v in np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=2))))
        d = int(rng.choice(dims))
        ox, oy = int(rng.integers(0, hi - N + 1)), int(rng.integers(0, hi - M + 1))
        F, K, G, L = pools[d]
        out.append(dict(rid=i, t=float(t[i]), key=f"market{i}", F=F[ox:ox + N], K=K[ox:ox + N],
                        G=G[oy:oy + M], L=L[oy:oy + M], n=_capacities(rng, N, "uniform1to3"),
                        m=_capacities(rng, M, "uniform1to3"), sigma=sigma, resolve=False))
    return out


def serving_request_sizes(count: int, rate: float = 200.0, lo: int = 1000, hi: int = 200_000,
                          seed: int = 1004) -> list:
    """Poisson arrival times and log-uniform sizes of a stream of solve requests."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    ln = rng.uniform(math.log(lo), math.log(hi), size=(count, 2))
    sizes = np.rint(np.exp(ln)).astype(np.int64)
    d = rng.choice([32, 64], size=count)
    resolve = rng.random(count) < 0.3
    return [dict(t=float(ti), N=int(a), M=int(b), d=int(di), resolve=bool(r))
            for ti, (a, b), di, r in zip(t, sizes, d, resolve)]


def crowding_market(N: int = 1000, M: int = 500, lam: float = 0.5, d: int = 32, sigma: float = 1.0,
                    seed: int = 1006):
    """A market with controlled preference crowding (Sec. 4.1's synthetic
    experiment: 1,000 candidates, 500 employers, crowding lambda in
    {0, 0.25, 0.5, 0.75}, beta = 1). Reading of its generator (the paper
    describes it in words): the probability that candidate x likes employer y
    interpolates an independent uniform draw and a value that falls with the
    employer's index, p_xy = (1 - lambda) U_xy + lambda (1 - y / M), and
    likewise q_yx = (1 - lambda) U'_yx + lambda (1 - x / N) for the employer's
    side; lambda = 0 is no crowding, larger lambda concentrates everyone's
    preferences on the same low-index users. The matching model's factors are
    the best rank-d approximations of the two preference matrices (truncated
    SVD, standing in for the paper's implicit-ALS fit to sampled
    interactions): F G^T ~ P, K L^T ~ Q^T, so phi = <f_x, g_y> + <k_x, l_y>.
    Returns (Market with float32 factors, P (N x M), Q (M x N)), P and Q in
    float64."""
    rng = np.random.default_rng(seed)
    P = (1.0 - lam) * rng.random((N, M)) + lam * (1.0 - np.arange(M) / M)[None, :]
    Q = (1.0 - lam) * rng.random((M, N)) + lam * (1.0 - np.arange(N) / N)[None, :]

    def rank_d(A):
        Uu, s, Vt = np.linalg.svd(A, full_matrices=False)
        r = np.sqrt(s[:d])
        return (Uu[:, :d] * r).astype(np.float32), (Vt[:d].T * r).astype(np.float32)

    F, G = rank_d(P)        # F G^T ~ P      (N x d, M x d)
    L, K = rank_d(Q)        # L K^T ~ Q, so K L^T ~ Q^T
    mk = Market(F, K, G, L, None, None, np.ones(N), np.ones(M), float(sigma), "fp32", seed,
                f"crowding N={N} M={M} lambda={lam} d={d}")
    return mk, P, Q
