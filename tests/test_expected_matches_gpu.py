"""Expected matches of the library's ranked lists on crowding markets (GPU).

Sec. 4.1's synthetic experiment: 1,000 candidates, 500 employers, crowding
lambda in {0, 0.75}, beta = 1. The market is solved and both sides' top-20
lists come from the library (tu_topk_partners); their expected number of
matches under the position-based model (v(k) = 1 / exp(k - 1)) from the
product's evaluation equals the oracle's double loop on the same lists, and
the lists at the ranking-stability stop give nearly the same expected matches
as the lists at the fixed point.
"""

import numpy as np
import pytest

import oracle
from paper_2411_19214_gb300 import evaluate
from synth import crowding_market

pytestmark = pytest.mark.gpu


def _lists(mkt, k):
    ix, _ = mkt.topk(0, k)
    iy, _ = mkt.topk(1, k)
    return ix.cpu().numpy(), iy.cpu().numpy()


@pytest.mark.parametrize("lam", [0.0, 0.75])
def test_expected_matches_of_library_lists(gpu_lib, lam):
    tu = gpu_lib
    mk, P, Q = crowding_market(1000, 500, lam=lam, d=32, sigma=1.0, seed=1006)
    mkt = tu.from_synth(mk)
    try:
        info = mkt.solve(tol=1e-6, max_iter=2000)
        assert info["converged"], info
        ix, iy = _lists(mkt, 20)
        em = evaluate.expected_matches(ix, iy, P, Q)
        ref = oracle.expected_matches(P, Q, ix.tolist(), iy.tolist())
        assert em == pytest.approx(ref, rel=1e-12)
        stop = tu.from_synth(mk)
        try:
            st = stop.solve_ranking(k=20, sample=1000, check_every=1, patience=2, max_iter=2000)
            assert st["converged"], st
            sx, sy = _lists(stop, 20)
            em_stop = evaluate.expected_matches(sx, sy, P, Q)
        finally:
            stop.close()
        print(f"lambda {lam}: expected matches {em:.4f} at the fixed point ({info['sweeps']} sweeps), "
              f"{em_stop:.4f} at the ranking stop ({st['sweeps']} sweeps)")
        assert abs(em_stop - em) <= 1e-2 * em
    finally:
        mkt.close()
