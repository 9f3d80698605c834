"""GPU tests of the ranking-stability stopping rule (the early-stopping
criterion the paper proposes for practical use: stop when the ranked lists of
both sides no longer change). The lists at the stop must be the lists of the
exact fixed point wherever the fixed point's scores are separated, and the
stop must come before the marginal residual reaches a tight tolerance."""

import numpy as np
import pytest

import oracle
from synth import make_market

from _parity import oracle_solve

pytestmark = pytest.mark.gpu

EPS = 1e-3  # score gap (natural log) above which the order at the stop must match the fixed point


def _ranked(lmu, k):
    return np.argsort(-lmu, axis=1, kind="stable")[:, :k]


def _separated(lmu, k):
    s = -np.sort(-lmu, axis=1)[:, :k + 1]
    gap = s[:, :-1] - s[:, 1:]
    ok = gap > EPS
    ok[:, 1:] &= gap[:, :-1] > EPS
    return ok


@pytest.mark.parametrize("path", ["fused", "dense"])
def test_stop_lists_equal_fixed_point_lists(gpu_lib, path):
    tu = gpu_lib
    mk = make_market(500, 450, 32, sigma=1.0, seed=77, bias_y=True, m_kind="uniform1to3",
                     dtype="bf16" if path == "fused" else "fp32")
    mkt = tu.from_synth(mk, path=path)
    try:
        info = mkt.solve_ranking(k=10, sample=100000, check_every=2, patience=3, max_iter=5000)
        assert info["converged"], info
        ix, _ = mkt.topk(0, 10)
        iy, _ = mkt.topk(1, 10)
        r, logA, f = oracle_solve(mk)
        lmu = oracle.log_mu(logA, r["log_u"], r["log_v"])
        for got, scores in ((ix.cpu().numpy(), lmu), (iy.cpu().numpy(), lmu.T)):
            want = _ranked(scores, 10)
            ok = _separated(scores, 10)
            assert np.all(got[ok] == want[ok])
        # the stop comes no later than a tight solve (1e-6: the FP32 floor of
        # the fused path's residual is a few 1e-7) plus the `patience` passing
        # checks the rule waits for once the lists have settled
        tight = tu.from_synth(mk, path=path)
        try:
            full = tight.solve(tol=1e-6, max_iter=20000)
            assert full["converged"] and info["sweeps"] <= full["sweeps"] + 2 * 3 + 2, (info, full)
        finally:
            tight.close()
    finally:
        mkt.close()


def test_stop_on_slow_market_and_arguments(gpu_lib):
    tu = gpu_lib
    # balanced with popularity biases: with Eq. iteration (translation step
    # off) thousands of sweeps to 1e-6, rankings settle far earlier
    mk = make_market(400, 400, 32, sigma=0.5, seed=5, bias_x=True, bias_y=True)
    mkt = tu.from_synth(mk)
    try:
        mkt.set_translation(False)
        info = mkt.solve_ranking(k=5, sample=400, check_every=5, patience=4, max_iter=20000)
        assert info["converged"] and info["residual_inf"] > 1e-6, info
        tight = mkt.solve(tol=1e-6, max_iter=50000, warm_start=True)
        assert tight["converged"] and tight["sweeps"] > info["sweeps"], (info, tight)
        cap = tu.tu_ipfp_solve_ranking(mkt.handle, 5, 400, 5, 4, 3)
        assert cap["status"] == tu.TU_ERR_NOT_CONVERGED and cap["sweeps"] == 3
        for bad in ((0, 10, 1, 1, 10), (64, 10, 1, 1, 10), (5, 0, 1, 1, 10), (5, 10, 0, 1, 10), (5, 10, 1, 0, 10),
                    (5, 10, 1, 1, -1)):
            with pytest.raises(tu.TuError) as e:
                tu.tu_ipfp_solve_ranking(mkt.handle, *bad)
            assert e.value.status == tu.TU_ERR_INVALID_ARG
    finally:
        mkt.close()
