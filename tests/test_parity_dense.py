"""GPU parity of the dense (materialised FP32 kernel) path against the FP64 oracle.

Tolerance (derivation): A-hat is FP32 (relative error ~1e-7 from the FP32 dot
product and expf), row sums are FP32 warp-tree sums of float4 partials, column
sums add FP32 chunk partials in FP64: log s is within ~1e-6, so one sweep moves
the log potentials by at most ~1e-6; ATOL_LOG = 1e-5. At the fixed point the
benchmark's FP32 bar applies: 1e-5 relative on mu and on the marginals.
"""

import numpy as np
import pytest

import oracle
from synth import dense_job_market, make_market, plain_dense_market

from _parity import dense_logA, oracle_solve, oracle_sweeps

pytestmark = pytest.mark.gpu

ATOL_LOG = 1e-5
MU_RTOL_FP32 = 1e-5


SHAPES = [(700, 555, 32), (1, 333, 8), (333, 1, 8), (2048, 1001, 32), (97, 4099, 5)]


@pytest.mark.parametrize("translate", [True, False], ids=["translated", "plain"])
@pytest.mark.parametrize("N,M,d", SHAPES, ids=lambda v: str(v))
def test_sweeps_match_oracle(gpu_lib, N, M, d, translate):
    tu = gpu_lib
    mk = make_market(N, M, d, sigma=0.5, seed=N + 3 * M, bias_y=True, m_kind="uniform1to5", dtype="fp32")
    mkt = tu.from_synth(mk, path="dense")
    try:
        mkt.set_translation(translate)
        done = 0
        for target in (1, 3, 8):
            mkt.sweep(target - done)
            done = target
            lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
            ou, ov = oracle_sweeps(mk, target, translate=translate)
            np.testing.assert_allclose(lu, ou, rtol=0, atol=ATOL_LOG, err_msg=f"log u after {target} sweeps")
            np.testing.assert_allclose(lv, ov, rtol=0, atol=ATOL_LOG, err_msg=f"log v after {target} sweeps")
    finally:
        mkt.close()


def test_job_market_solve_matches_oracle(gpu_lib):
    """Job-market recipe (lognormal job popularity, capacities U{1..5}, sigma 0.5)
    at a size the oracle solves in seconds."""
    tu = gpu_lib
    mk = dense_job_market(N=2000, M=1000)
    mkt = tu.from_synth(mk, path="dense")
    try:
        # tol of the job-market configuration; the FP32 row sums put the
        # residual floor near 1e-7 (relative error of s), so 1e-6 is reachable
        info = mkt.solve(tol=1e-6, max_iter=2000)
        assert info["residual_inf"] <= 1e-6
        assert info["converged"], info
        r, logA, f = oracle_solve(mk)
        mu_ref = np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))
        mu = mkt.mu_block().double().cpu().numpy()
        rel = np.max(np.abs(mu / mu_ref - 1))
        print(f"dense job market: max rel mu err {rel:.3e}, sweeps {info['sweeps']}")
        np.testing.assert_allclose(mu, mu_ref, rtol=MU_RTOL_FP32, atol=0)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        # marginals (constraints of Eq. primary optimization) of the GPU solution
        np.testing.assert_allclose(mu.sum(1) + np.exp(2 * lu), f["n"], rtol=MU_RTOL_FP32)
        np.testing.assert_allclose(mu.sum(0) + np.exp(2 * lv), f["m"], rtol=MU_RTOL_FP32)
        cx = oracle.match_count(f["n"], r["log_u"])
        assert abs(info["match_count"] - cx) <= MU_RTOL_FP32 * cx
    finally:
        mkt.close()


def test_plain_balanced_market_fixed_point(gpu_lib):
    """Plain balanced market (factors N(0, 1/d), unit capacities, sigma 1),
    reduced to 300 x 300 so the oracle converges in seconds."""
    tu = gpu_lib
    mk = plain_dense_market(N=300, M=300)
    mkt = tu.from_synth(mk, path="dense")
    try:
        info = mkt.solve(tol=1e-6, max_iter=20000)
        assert info["converged"], info
        r, logA, f = oracle_solve(mk, tol=1e-12)
        mu_ref = np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))
        mu = mkt.mu_block().double().cpu().numpy()
        rel = np.max(np.abs(mu / mu_ref - 1))
        cx = oracle.match_count(f["n"], r["log_u"])
        print(f"balanced 300: max rel mu err {rel:.3e}; match {info['match_count']:.9f} vs {cx:.9f}")
        # a residual of 1e-6 in a balanced market (slow mode ~ N) bounds mu only to ~N * 1e-6
        np.testing.assert_allclose(mu, mu_ref, rtol=3e-4)
        assert abs(info["match_count"] - cx) <= 1e-5 * cx
    finally:
        mkt.close()


def test_full_size_job_market_sampled(gpu_lib):
    """20000 x 10000, d = 32: three sweeps on the GPU, then one more sweep
    checked on 64 sampled rows and columns against the oracle's update from
    the GPU's own state (translation step off: one sweep of Eq. iteration)."""
    tu = gpu_lib
    mk = dense_job_market()
    mkt = tu.from_synth(mk, path="dense")
    try:
        mkt.set_translation(False)
        mkt.sweep(3)
        lu0, lv0 = (t.double().cpu().numpy() for t in mkt.potentials())
        mkt.sweep(1)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        rng = np.random.default_rng(1)
        rows = np.sort(rng.choice(mk.N, 64, replace=False))
        cols = np.sort(rng.choice(mk.M, 64, replace=False))
        f = mk.f64()
        _, ou = oracle.sampled_row_update(mk.F, mk.K, mk.G, mk.L, f["sigma"], f["n"], lv0, rows, None, mk.bias_y)
        np.testing.assert_allclose(lu[rows], ou, atol=ATOL_LOG)
        _, ov = oracle.sampled_row_update(mk.G, mk.L, mk.F, mk.K, f["sigma"], f["m"], lu, cols, mk.bias_y, None)
        np.testing.assert_allclose(lv[cols], ov, atol=ATOL_LOG)
    finally:
        mkt.close()


@pytest.mark.parametrize("N,M", [(70_000, 2_000), (2_000, 70_000)])
def test_many_rows_per_cta_sampled(gpu_lib, N, M):
    """Tall and wide markets: one of the two passes gives every CTA more than
    two blocks of 32 rows, so the row pass reuses its double-buffered blocks
    of parked row sums (the path a 20,000-row pass does not reach). Two
    sweeps, then one more checked on sampled rows and columns (the first and
    last rows included) against the oracle's update from the GPU's own state
    (translation step off: one sweep of Eq. iteration)."""
    tu = gpu_lib
    mk = make_market(N, M, 16, sigma=0.5, seed=N + 7, bias_y=True, m_kind="uniform1to5", dtype="fp32")
    mkt = tu.from_synth(mk, path="dense")
    try:
        mkt.set_translation(False)
        mkt.sweep(2)
        lu0, lv0 = (t.double().cpu().numpy() for t in mkt.potentials())
        mkt.sweep(1)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        rng = np.random.default_rng(2)
        rows = np.unique(np.r_[0, N - 1, rng.choice(N, 62, replace=False)])
        cols = np.unique(np.r_[0, M - 1, rng.choice(M, 62, replace=False)])
        f = mk.f64()
        _, ou = oracle.sampled_row_update(mk.F, mk.K, mk.G, mk.L, f["sigma"], f["n"], lv0, rows, None, mk.bias_y)
        np.testing.assert_allclose(lu[rows], ou, atol=ATOL_LOG)
        _, ov = oracle.sampled_row_update(mk.G, mk.L, mk.F, mk.K, f["sigma"], f["m"], lu, cols, mk.bias_y, None)
        np.testing.assert_allclose(lv[cols], ov, atol=ATOL_LOG)
        assert np.all(np.isfinite(lu)) and np.all(np.isfinite(lv))
    finally:
        mkt.close()


def test_tall_market_beyond_one_grid_height(gpu_lib):
    """4,300,000 x 8: more row tiles of 64 than one grid's height (65,535)
    holds, so building A-hat strides over row tiles, and a 600,000-row mu
    block has more than 65,535 blocks of 8 rows. Two sweeps, then one more
    checked on sampled rows (both sides of the grid-height bound and the last
    row included) and on every column against the oracle's update from the
    GPU's own state; then the mu block of the last 600,000 rows (translation
    step off: one sweep of Eq. iteration)."""
    tu = gpu_lib
    N, M = 4_300_000, 8
    assert (N + 63) // 64 > 65535
    mk = make_market(N, M, 4, sigma=0.5, seed=29, bias_y=True, m_kind="uniform1to5", dtype="fp32")
    mkt = tu.from_synth(mk, path="dense")
    try:
        mkt.set_translation(False)
        mkt.sweep(2)
        lu0, lv0 = (t.double().cpu().numpy() for t in mkt.potentials())
        mkt.sweep(1)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        rng = np.random.default_rng(3)
        edge = 64 * 65535
        rows = np.unique(np.r_[0, edge - 1, edge, edge + 63, N - 1, rng.choice(N, 59, replace=False)])
        f = mk.f64()
        _, ou = oracle.sampled_row_update(mk.F, mk.K, mk.G, mk.L, f["sigma"], f["n"], lv0, rows, None, mk.bias_y)
        np.testing.assert_allclose(lu[rows], ou, atol=ATOL_LOG)
        _, ov = oracle.sampled_row_update(mk.G, mk.L, mk.F, mk.K, f["sigma"], f["m"], lu, np.arange(M), mk.bias_y,
                                          None)
        # a column sum runs over 4.3e6 terms: each of the pass's 1,024
        # accumulators is a compensated (Kahan) FP32 sum of about N / 1024
        # terms, so the column update meets the FP32 bar like a short row; a
        # row tile left unbuilt would move log v by about 0.025
        col_err = float(np.max(np.abs(lv - ov)))
        row_err = float(np.max(np.abs(lu[rows] - ou)))
        print(f"4.3e6 x 8: max |log u - oracle| {row_err:.2e} (sampled rows), max |log v - oracle| {col_err:.2e}")
        np.testing.assert_allclose(lv, ov, atol=ATOL_LOG)
        nx = 600_000
        x0 = N - nx
        mu = mkt.mu_block(x0, nx, 0, M).double().cpu().numpy()
        Phi = oracle.phi_dense(f["F"][x0:], f["K"][x0:], f["G"], f["L"], None, f["bias_y"])
        ref = np.exp(oracle.log_mu(oracle.log_kernel(Phi, f["sigma"]), lu[x0:], lv))
        np.testing.assert_allclose(mu, ref, rtol=MU_RTOL_FP32)
    finally:
        mkt.close()
