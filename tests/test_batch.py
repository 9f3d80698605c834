"""GPU tests of the batched launch: many independent markets swept by one
persistent tensor-core launch per half-sweep (tu_batch_*).

Each market of a batch runs the arithmetic of its own sweep (Eq.
iteration_minibatch): the same partner shift and FP32 partner vector, the same
own tiles reduced by the same epilogue. So after k batched sweeps its
potentials must equal, bit for bit, k sweeps of the same market alone, and the
fused-path tolerances against the FP64 oracle apply (ATOL_LOG, derived in
test_parity_fused.py). Only the FP64 residual sums are reduced in another
order; their maximum part is exact.
"""

import numpy as np
import pytest
import torch

import oracle
from synth import batched_markets, make_market

from _parity import oracle_solve, oracle_sweeps

pytestmark = pytest.mark.gpu

ATOL_LOG = 2e-5
MU_RTOL_BF16 = 1e-3
MATCH_RTOL = 1e-5

# ragged and degenerate shapes (one own tile, many, a single user per side),
# all with 2d <= 64 so they share one packed width
SHAPES = [(700, 555, 32), (256, 128, 32), (1, 300, 24), (300, 1, 24), (5, 7, 1), (1000, 333, 32),
          (2049, 130, 30), (130, 2049, 32), (513, 257, 16)]


def _mk(N, M, d, seed, **kw):
    base = dict(sigma=0.5, bias_x=True, bias_y=True, n_kind="uniform_real", m_kind="uniform_real", dtype="bf16")
    base.update(kw)
    return make_market(N, M, d, seed=seed, **base)


def _pot(mkt):
    lu, lv = mkt.potentials()
    return lu.cpu(), lv.cpu()


def test_batch_sweeps_bit_identical_to_single_and_match_oracle(gpu_lib):
    tu = gpu_lib
    mks = [_mk(N, M, d, seed=31 + i) for i, (N, M, d) in enumerate(SHAPES)]
    alone = [tu.from_synth(mk) for mk in mks]
    grouped = [tu.from_synth(mk) for mk in mks]
    batch = tu.Batch(grouped)
    try:
        batch.sweep(3)
        torch.cuda.synchronize()
        for mkt in alone:
            mkt.sweep(3)
        for i, (a, b) in enumerate(zip(alone, grouped)):
            (au, av), (bu, bv) = _pot(a), _pot(b)
            assert torch.equal(au, bu) and torch.equal(av, bv), f"market {i} {SHAPES[i]} differs from its solo sweeps"
        # residual of the returned state: per-row values are identical, the max is exact
        res_b = batch.sweep(2, residual=True)
        res_a = np.array([mkt.sweep(2, residual=True) for mkt in alone])
        np.testing.assert_array_equal(res_b, res_a)
        for i, (mk, mkt) in enumerate(zip(mks, grouped)):
            lu, lv = (t.double().numpy() for t in _pot(mkt))
            ou, ov = oracle_sweeps(mk, 5)
            np.testing.assert_allclose(lu, ou, rtol=0, atol=ATOL_LOG, err_msg=f"log u, market {i}")
            np.testing.assert_allclose(lv, ov, rtol=0, atol=ATOL_LOG, err_msg=f"log v, market {i}")
    finally:
        batch.close()
        for mkt in alone + grouped:
            mkt.close()


def test_batch_solve_matches_oracle_fixed_points(gpu_lib):
    tu = gpu_lib
    # with Eq. iteration (translation step off) unbalanced markets converge in
    # tens of sweeps, the near-balanced one in hundreds: the fast ones leave
    # the launch early
    shapes = [(400, 900, 32), (900, 400, 32), (300, 330, 32), (64, 1000, 16), (1200, 700, 32)]
    mks = [_mk(N, M, d, seed=101 + i, sigma=1.0, bias_x=False, bias_y=(i % 2 == 0), n_kind="uniform1to3",
               m_kind="unit") for i, (N, M, d) in enumerate(shapes)]
    mkts = [tu.from_synth(mk) for mk in mks]
    for mkt in mkts:
        mkt.set_translation(False)
    batch = tu.Batch(mkts)
    try:
        st, infos = batch.solve(tol=1e-6, max_iter=20000)
        assert st == tu.TU_OK, infos
        assert len({i["sweeps"] for i in infos}) > 1, "markets should stop at different sweep counts"
        for mk, mkt, info in zip(mks, mkts, infos):
            assert info["converged"] and info["residual_inf"] <= 1e-6, info
            r, logA, f = oracle_solve(mk)
            mu_ref = np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))
            mu = mkt.mu_block().double().cpu().numpy()
            np.testing.assert_allclose(mu, mu_ref, rtol=MU_RTOL_BF16, atol=0, err_msg=mk.recipe)
            cx = oracle.match_count(f["n"], r["log_u"])
            assert abs(info["match_count"] - cx) <= MATCH_RTOL * cx, (info, cx)
    finally:
        batch.close()
        for mkt in mkts:
            mkt.close()


def test_batch_solve_state_equals_solo_sweeps(gpu_lib):
    """A market's state after a batched solve is that of the same number of
    solo sweeps: markets that leave the launch are not touched afterwards."""
    tu = gpu_lib
    shapes = [(500, 800, 32), (700, 300, 32), (260, 270, 24)]
    mks = [_mk(N, M, d, seed=7 + i, sigma=1.0, bias_x=False, bias_y=False, n_kind="unit", m_kind="unit")
           for i, (N, M, d) in enumerate(shapes)]
    mkts = [tu.from_synth(mk) for mk in mks]
    batch = tu.Batch(mkts)
    try:
        st, infos = batch.solve(tol=1e-5, max_iter=5000)
        assert st == tu.TU_OK, infos
        for mk, mkt, info in zip(mks, mkts, infos):
            solo = tu.from_synth(mk)
            try:
                solo.sweep(info["sweeps"])
                (au, av), (bu, bv) = _pot(solo), _pot(mkt)
                assert torch.equal(au, bu) and torch.equal(av, bv), (mk.recipe, info)
            finally:
                solo.close()
        # warm start from converged potentials: every market is certified
        # before any sweep and its state is left as it was
        before = [_pot(m) for m in mkts]
        st2, infos2 = batch.solve(tol=1e-5, max_iter=5000, warm_start=True)
        assert st2 == tu.TU_OK and all(i["sweeps"] == 0 for i in infos2), infos2
        for (au, av), mkt in zip(before, mkts):
            bu, bv = _pot(mkt)
            assert torch.equal(au, bu) and torch.equal(av, bv)
    finally:
        batch.close()
        for mkt in mkts:
            mkt.close()


def test_batch_not_converged_reports_per_market(gpu_lib):
    tu = gpu_lib
    mks = [_mk(300, 900, 32, seed=1, sigma=1.0, bias_x=False, bias_y=False, n_kind="unit", m_kind="unit"),
           _mk(600, 600, 32, seed=2, sigma=1.0, bias_x=True, bias_y=True, n_kind="unit", m_kind="unit")]
    mkts = [tu.from_synth(mk) for mk in mks]
    for mkt in mkts:
        mkt.set_translation(False)  # Eq. iteration: the balanced market is slow
    batch = tu.Batch(mkts)
    try:
        st, infos = batch.solve(tol=1e-6, max_iter=40)
        assert st == tu.TU_ERR_NOT_CONVERGED
        assert infos[0]["converged"], infos[0]          # unbalanced: fast
        assert not infos[1]["converged"] and infos[1]["sweeps"] == 40  # balanced with biases: slow
        assert infos[1]["residual_inf"] > 1e-6
    finally:
        batch.close()
        for mkt in mkts:
            mkt.close()


def test_batch_auto_relaxation_same_fixed_point(gpu_lib):
    tu = gpu_lib
    mk = _mk(800, 800, 32, seed=17, sigma=1.0, bias_x=False, bias_y=False, n_kind="unit", m_kind="unit")
    other = _mk(300, 1000, 32, seed=18, sigma=1.0, bias_x=False, bias_y=False, n_kind="unit", m_kind="unit")
    plain = tu.from_synth(mk)
    relaxed = [tu.from_synth(mk), tu.from_synth(other)]
    for m in [plain] + relaxed:
        m.set_translation(False)  # relaxation against Eq. iteration itself
    for m in relaxed:
        m.set_relaxation(0.0)
    batch = tu.Batch(relaxed)
    try:
        ip = plain.solve(tol=1e-6, max_iter=20000)
        st, infos = batch.solve(tol=1e-6, max_iter=20000)
        assert ip["converged"] and st == tu.TU_OK, (ip, infos)
        assert infos[0]["sweeps"] < ip["sweeps"], (infos[0], ip)
        r, logA, f = oracle_solve(mk)
        mu_ref = np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))
        mu = relaxed[0].mu_block().double().cpu().numpy()
        np.testing.assert_allclose(mu, mu_ref, rtol=MU_RTOL_BF16, atol=0)
    finally:
        batch.close()
        for m in [plain] + relaxed:
            m.close()


def test_batch_translated_solve_matches_oracle_fixed_points(gpu_lib):
    """With the translation step (the default), balanced and unbalanced
    markets with and without popularity biases all reach tol in a few sweeps,
    at the oracle's fixed points; each market's state equals that many solo
    sweeps bit for bit."""
    tu = gpu_lib
    shapes = [(600, 600, 32), (400, 900, 32), (900, 400, 32), (1000, 1000, 16), (64, 1000, 16)]
    mks = [_mk(N, M, d, seed=201 + i, sigma=0.5, bias_x=(i % 2 == 0), bias_y=True, n_kind="unit", m_kind="unit")
           for i, (N, M, d) in enumerate(shapes)]
    mkts = [tu.from_synth(mk) for mk in mks]
    batch = tu.Batch(mkts)
    try:
        st, infos = batch.solve(tol=1e-6, max_iter=2000)
        assert st == tu.TU_OK, infos
        for mk, mkt, info in zip(mks, mkts, infos):
            assert info["converged"] and info["sweeps"] <= 40, (mk.recipe, info)
            r, logA, f = oracle_solve(mk)
            mu_ref = np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))
            mu = mkt.mu_block().double().cpu().numpy()
            np.testing.assert_allclose(mu, mu_ref, rtol=MU_RTOL_BF16, atol=0, err_msg=mk.recipe)
            cx = oracle.match_count(f["n"], r["log_u"])
            assert abs(info["match_count"] - cx) <= MATCH_RTOL * cx, (info, cx)
            solo = tu.from_synth(mk)
            try:
                solo.sweep(info["sweeps"])
                (au, av), (bu, bv) = _pot(solo), _pot(mkt)
                assert torch.equal(au, bu) and torch.equal(av, bv), (mk.recipe, info)
            finally:
                solo.close()
    finally:
        batch.close()
        for mkt in mkts:
            mkt.close()


def test_batch_invalid_arguments(gpu_lib):
    tu = gpu_lib
    a = tu.from_synth(_mk(100, 120, 32, seed=3))
    b64 = tu.from_synth(_mk(100, 120, 64, seed=4))
    dense = tu.from_synth(_mk(100, 120, 32, seed=5, dtype="fp32"), path="dense")
    try:
        for handles in ([], [a.handle, b64.handle], [a.handle, a.handle], [dense.handle]):
            with pytest.raises(tu.TuError) as e:
                tu.tu_batch_create(handles)
            assert e.value.status == tu.TU_ERR_INVALID_ARG
        batch = tu.Batch([a])
        with pytest.raises(tu.TuError) as e:
            batch.sweep(-1)
        assert e.value.status == tu.TU_ERR_INVALID_ARG
        with pytest.raises(tu.TuError) as e:
            batch.solve(tol=-1.0, max_iter=10)
        assert e.value.status == tu.TU_ERR_INVALID_ARG
        batch.close()
    finally:
        for m in (a, b64, dense):
            m.close()


def test_batched_workload_full_size_sampled(gpu_lib):
    """The 512-market workload the benchmark times (sizes log-uniform in
    [100, 50,000], d = 32): one batched sweep; for a sample of markets
    (including the largest) the oracle recomputes sampled rows of the X
    half-sweep from u = v = 1 and sampled columns of the Y half-sweep from the
    device's new log u; four markets are compared bit for bit with solo sweeps.
    The translation step is off (one sweep of Eq. iteration)."""
    tu = gpu_lib
    mks = batched_markets()
    mkts = [tu.from_synth(mk) for mk in mks]
    for mkt in mkts:
        mkt.set_translation(False)
    batch = tu.Batch(mkts)
    rng = np.random.default_rng(5)
    try:
        res = batch.sweep(1, residual=True)
        assert np.all(np.isfinite(res))
        pairs = np.array([mk.N * mk.M for mk in mks])
        sample = sorted({int(np.argmax(pairs)), int(np.argmin(pairs))} | set(rng.choice(len(mks), 4, replace=False)))
        for i in sample:
            mk, mkt = mks[i], mkts[i]
            f = mk.f64()
            lu, lv = (t.double().numpy() for t in _pot(mkt))
            rows = rng.choice(mk.N, min(mk.N, 300), replace=False)
            cols = rng.choice(mk.M, min(mk.M, 300), replace=False)
            _, ou = oracle.sampled_row_update(mk.F, mk.K, mk.G, mk.L, f["sigma"], f["n"], np.zeros(mk.M), rows)
            _, ov = oracle.sampled_row_update(mk.G, mk.L, mk.F, mk.K, f["sigma"], f["m"], lu, cols)
            np.testing.assert_allclose(lu[rows], ou, rtol=0, atol=ATOL_LOG, err_msg=f"market {i} rows")
            np.testing.assert_allclose(lv[cols], ov, rtol=0, atol=ATOL_LOG, err_msg=f"market {i} cols")
        for i in sample[:4]:
            solo = tu.from_synth(mks[i])
            try:
                solo.set_translation(False)
                solo.sweep(1)
                (au, av), (bu, bv) = _pot(solo), _pot(mkts[i])
                assert torch.equal(au, bu) and torch.equal(av, bv), mks[i].recipe
            finally:
                solo.close()
    finally:
        batch.close()
        for mkt in mkts:
            mkt.close()
