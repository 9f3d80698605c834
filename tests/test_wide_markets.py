"""Markets whose factor range exceeds one shift per half-sweep (GPU).

With max|a_x| max|b_y| / (2 sigma) above 40 (strong preferences, small
sigma), one shift per half-sweep would leave FP32 exponents out of range; the
fused path then keeps a running maximum of every own row's exponents
c phi_hat + g and rescales the row's sum by an exact power of two whenever it
grows, so that no term exceeds 2^0 (tu_market_create). These markets are
checked against the oracle on the same rounded factors.

Tolerance (derived): the tensor cores accumulate phi = <a, b> of exact BF16
products in FP32; over the 2d = 128 terms the rounding is about
sqrt(2d) 2^-24 max|a| max|b| absolute, and the exponent multiplies it by
1 / (2 sigma). At the bound B = max|a| max|b| / (2 sigma) this is
B sqrt(2d) 2^-24 per term (about 1.4e-4 for the market below, B ~ 200), three
orders above the narrow markets' 1e-7; a log potential, a log row sum of
such terms, moves by at most that. The tests allow 4 B sqrt(2d) 2^-24 plus
the narrow path's 2e-5.
"""

import math

import numpy as np
import pytest

import oracle
from synth import make_market

from _parity import dense_logA, oracle_solve, oracle_sweeps

pytestmark = pytest.mark.gpu


def _mk(N=700, M=555, d=64, sigma=0.01, seed=33):
    return make_market(N, M, d, sigma=sigma, seed=seed, bias_x=True, bias_y=True, n_kind="uniform_real",
                       m_kind="uniform_real", dtype="bf16")


def _bound(mk):
    a = np.sqrt(np.sum(mk.F.astype(np.float64) ** 2, 1) + np.sum(mk.K.astype(np.float64) ** 2, 1)).max()
    b = np.sqrt(np.sum(mk.G.astype(np.float64) ** 2, 1) + np.sum(mk.L.astype(np.float64) ** 2, 1)).max()
    return a * b / (2.0 * mk.sigma)


def _atol(mk):
    return 2e-5 + 4.0 * _bound(mk) * math.sqrt(2 * mk.d) * 2.0 ** -24


def test_wide_market_sweeps_match_oracle(gpu_lib):
    tu = gpu_lib
    mk = _mk()
    assert _bound(mk) > 100.0  # far beyond the single-shift limit of 40
    atol = _atol(mk)
    mkt = tu.from_synth(mk)
    try:
        done = 0
        errs = []
        for target in (1, 2, 5):
            mkt.sweep(target - done)
            done = target
            lu, lv = mkt.potentials64()
            ou, ov = oracle_sweeps(mk, target)
            errs.append(max(np.abs(lu - ou).max(), np.abs(lv - ov).max()))
            np.testing.assert_allclose(lu, ou, rtol=0, atol=atol, err_msg=f"log u after {target} sweeps")
            np.testing.assert_allclose(lv, ov, rtol=0, atol=atol, err_msg=f"log v after {target} sweeps")
        print(f"wide market (bound {_bound(mk):.0f}): max |log potential error| {max(errs):.2e}, allowed {atol:.2e}")
    finally:
        mkt.close()


@pytest.mark.parametrize("order", ["ascending", "descending"])
def test_running_maximum_across_column_orders(gpu_lib, order):
    """The running maximum under its two extremes. With the partner side sorted
    by bias ascending, the exponents of a row tend to grow along its
    columns, so its shift rises in chunk after chunk and everything summed
    before is rescaled again and again; sorted descending, the first chunk
    holds the largest terms and the shift hardly moves. The permutation
    leaves the market's fixed point unchanged (Eq. iteration is equivariant
    under relabelling the partners), so both orders must match the oracle
    on the permuted market, and each other."""
    import dataclasses

    tu = gpu_lib
    base = _mk(N=300, M=1000, d=64, seed=37)
    perm = np.argsort(base.bias_y, kind="stable")
    if order == "descending":
        perm = perm[::-1].copy()
    mk = dataclasses.replace(base, G=base.G[perm], L=base.L[perm], bias_y=base.bias_y[perm], m=base.m[perm])
    assert _bound(mk) > 100.0
    atol = _atol(mk)
    mkt = tu.from_synth(mk)
    try:
        mkt.sweep(3)
        lu, lv = mkt.potentials64()
        ou, ov = oracle_sweeps(mk, 3)
        np.testing.assert_allclose(lu, ou, rtol=0, atol=atol)
        np.testing.assert_allclose(lv, ov, rtol=0, atol=atol)
        print(f"{order}: max |log potential error| {max(np.abs(lu - ou).max(), np.abs(lv - ov).max()):.2e}")
    finally:
        mkt.close()


def test_wide_market_solve_lists_and_mu(gpu_lib):
    """Solved to max(1e-6, 2 B 2^-24), the attainable residual: a row's
    dominant terms pair an exponent c phi of hundreds with a partner potential
    g of nearly the opposite size, both FP32, so their spacing (B 2^-24 in
    relative terms) moves a row sum between passes once the potentials shift
    by a rounding; mu and the match count
    against the oracle's fixed point within the derived tolerance; ranked lists
    of both sides equal the oracle's wherever its score gaps exceed it; mu
    blocks are representable although the exponents reach hundreds."""
    tu = gpu_lib
    mk = _mk(seed=34)
    atol = _atol(mk)
    mkt = tu.from_synth(mk)
    try:
        tol = max(1e-6, 2.0 * _bound(mk) * 2.0 ** -24)
        info = mkt.solve(tol=tol, max_iter=5000)
        assert info["converged"], info
        r, logA, f = oracle_solve(mk, tol=1e-12)
        lmu = oracle.log_mu(logA, r["log_u"], r["log_v"])
        mu = mkt.mu_block().double().cpu().numpy()
        assert np.all(np.isfinite(mu))
        rel = np.abs(mu / np.exp(lmu) - 1.0)
        # log mu = phi / (2 sigma) + log u + log v: three terms of the size above
        assert rel.max() <= 3.0 * atol + 1e-5, rel.max()
        cx = oracle.match_count(f["n"], r["log_u"])
        assert abs(info["match_count"] - cx) <= 3.0 * atol * cx
        for side, scores in ((0, lmu), (1, lmu.T)):
            idx, lm = mkt.topk(side, 10)
            idx, lm = idx.cpu().numpy(), lm.double().cpu().numpy()
            order = np.argsort(-scores, axis=1, kind="stable")
            eps = 4.0 * atol
            for row in range(idx.shape[0]):
                s_sorted = scores[row, order[row]]
                for i in range(10):
                    gap = min(s_sorted[i - 1] - s_sorted[i] if i else np.inf, s_sorted[i] - s_sorted[i + 1])
                    if gap > eps:
                        assert idx[row, i] == order[row, i], (side, row, i)
                    assert abs(lm[row, i] - scores[row, idx[row, i]]) <= eps
        print(f"wide market solved in {info['sweeps']} sweeps; mu rel err {rel.max():.2e}, "
              f"match {abs(info['match_count'] / cx - 1):.2e}")
    finally:
        mkt.close()


def test_wide_markets_refused_where_one_shift_is_needed(gpu_lib):
    """The dense path's FP32 A-hat and the batched kernel's one shift per
    market cannot take a wide market: TU_ERR_UNSUPPORTED."""
    tu = gpu_lib
    mk = _mk(N=200, M=150, d=16, sigma=0.005, seed=35)
    assert _bound(mk) > 40.0
    f32 = make_market(200, 150, 16, sigma=0.005, seed=35, dtype="fp32")
    with pytest.raises(tu.TuError) as e:
        tu.from_synth(f32, path="dense")
    assert e.value.status == tu.TU_ERR_UNSUPPORTED
    wide = tu.from_synth(mk)
    narrow = tu.from_synth(_mk(N=200, M=150, d=16, sigma=1.0, seed=36))
    try:
        with pytest.raises(tu.TuError) as e:
            tu.tu_batch_create([narrow.handle, wide.handle])
        assert e.value.status == tu.TU_ERR_UNSUPPORTED
    finally:
        wide.close()
        narrow.close()


@pytest.mark.parametrize("per", ["row", "side"])
def test_wide_fp8_market_sweeps_match_oracle(gpu_lib, per):
    """The wide path with e4m3 factors (per-row scales multiply the
    accumulator entries before the running maximum; per-side scales fold into c),
    against the oracle on the same quantized factors."""
    from synth import fp8_quantized
    tu = gpu_lib
    mk = make_market(600, 450, 64, sigma=0.01, seed=35, bias_x=True, bias_y=True, n_kind="uniform_real",
                     m_kind="uniform_real", dtype="fp32")
    q, _ = fp8_quantized(mk, per)
    assert _bound(q) > 100.0
    atol = _atol(q)
    mkt = tu.from_synth(mk, fp8="rows" if per == "row" else "side")
    try:
        mkt.sweep(3)
        lu, lv = mkt.potentials64()
        ou, ov = oracle_sweeps(q, 3)
        err = max(np.abs(lu - ou).max(), np.abs(lv - ov).max())
        print(f"\nwide FP8 ({per} scales, bound {_bound(q):.0f}): max |log potential error| {err:.2e}, allowed {atol:.2e}")
        assert err <= atol
    finally:
        mkt.close()
