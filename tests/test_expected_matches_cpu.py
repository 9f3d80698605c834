"""Expected number of matches of ranked lists (Sec. 4.1), on the CPU.

The oracle's definition is pinned by a 3 x 3 market worked by hand and by
planted mistakes (the examination function shifted by one position, one side's
examination dropped, the employers' like-probabilities transposed); the
product's vectorised evaluation (paper_2411_19214_gb300.evaluate) must equal
the oracle's double loop on random lists, mutual and one-sided entries mixed.
"""

import math

import numpy as np
import pytest

import oracle
from oracle import ipfp as O
from paper_2411_19214_gb300 import evaluate
from synth import crowding_market

# 3 candidates x 3 employers, every list complete (best first)
LISTS_X = [[0, 1, 2], [1, 0, 2], [2, 1, 0]]
LISTS_Y = [[0, 1, 2], [1, 2, 0], [0, 2, 1]]
P3 = np.array([[0.9, 0.5, 0.2], [0.4, 0.8, 0.1], [0.3, 0.6, 0.7]])   # P[x][y]: x likes y
Q3 = np.array([[0.6, 0.3, 0.5], [0.2, 0.9, 0.4], [0.7, 0.1, 0.8]])   # Q[y][x]: y likes x


def test_three_by_three_by_hand():
    """Positions (x's rank of y, y's rank of x) for every pair, from the lists:
    (0,0): 1,1  (0,1): 2,3  (0,2): 3,1
    (1,0): 2,2  (1,1): 1,1  (1,2): 3,3
    (2,0): 3,3  (2,1): 2,2  (2,2): 1,2
    so E = sum e^{-(kx-1)} e^{-(ky-1)} P[x][y] Q[y][x] =
      0.9*0.6 + e^-3*0.5*0.2 + e^-2*0.2*0.7
    + e^-2*0.4*0.3 + 0.8*0.9 + e^-4*0.1*0.1
    + e^-4*0.3*0.5 + e^-2*0.6*0.4 + e^-1*0.7*0.8."""
    e = math.exp
    want = (0.9 * 0.6 + e(-3) * 0.5 * 0.2 + e(-2) * 0.2 * 0.7
            + e(-2) * 0.4 * 0.3 + 0.8 * 0.9 + e(-4) * 0.1 * 0.1
            + e(-4) * 0.3 * 0.5 + e(-2) * 0.6 * 0.4 + e(-1) * 0.7 * 0.8)
    assert oracle.expected_matches(P3, Q3, LISTS_X, LISTS_Y) == pytest.approx(want, rel=1e-14)


def test_truncated_lists_count_only_mutual_entries():
    """With lists of length 1 only the pairs that list each other first count:
    (0,0) and (1,1) here; x2 lists y2, but y2 lists x0 first."""
    lx = [[0], [1], [2]]
    ly = [[0], [1], [0]]
    want = 0.9 * 0.6 + 0.8 * 0.9
    assert oracle.expected_matches(P3, Q3, lx, ly) == pytest.approx(want, rel=1e-14)


def _bad_shifted(P, Q, lists_x, lists_y):
    total = 0.0
    for x in range(len(lists_x)):
        for y in range(len(lists_y)):
            if y in lists_x[x] and x in lists_y[y]:
                kx, ky = list(lists_x[x]).index(y) + 1, list(lists_y[y]).index(x) + 1
                total += np.exp(-kx) * P[x][y] * np.exp(-ky) * Q[y][x]
    return total


def _bad_one_sided(P, Q, lists_x, lists_y):
    total = 0.0
    for x in range(len(lists_x)):
        for y in range(len(lists_y)):
            if y in lists_x[x] and x in lists_y[y]:
                kx = list(lists_x[x]).index(y) + 1
                total += np.exp(-(kx - 1)) * P[x][y] * Q[y][x]
    return total


_EXPECTED_MATCHES = O.expected_matches


def _bad_transposed(P, Q, lists_x, lists_y):
    return _EXPECTED_MATCHES(P, np.asarray(Q).T, lists_x, lists_y)


def test_planted_mistakes_are_caught(monkeypatch):
    for bad in (_bad_shifted, _bad_one_sided, _bad_transposed):
        with monkeypatch.context() as mp:
            mp.setattr(O, "expected_matches", bad)
            mp.setattr(oracle, "expected_matches", bad)
            with pytest.raises(AssertionError):
                test_three_by_three_by_hand()
    test_three_by_three_by_hand()


@pytest.mark.parametrize("N,M,k,seed", [(30, 20, 7, 1), (25, 40, 3, 2), (9, 11, 11, 3), (50, 50, 1, 4)])
def test_product_evaluation_equals_the_oracle(N, M, k, seed):
    rng = np.random.default_rng(seed)
    P = rng.random((N, M))
    Q = rng.random((M, N))
    idx_x = np.stack([rng.permutation(M)[:k] for _ in range(N)])
    idx_y = np.stack([rng.permutation(N)[:k] for _ in range(M)])
    # make some pairs mutual at the top so the sum is not tiny (lists keep
    # distinct entries, as ranked lists do)
    for i in range(min(N, M)):
        for lists, j in ((idx_x, i), (idx_y, i)):
            row = [v for v in lists[j] if v != i]
            lists[j] = np.array([i] + row[: k - 1])
    want = oracle.expected_matches(P, Q, idx_x.tolist(), idx_y.tolist())
    got = evaluate.expected_matches(idx_x, idx_y, P, Q)
    assert got == pytest.approx(want, rel=1e-12)
    assert want > 0.0


def test_crowding_generator():
    """lambda = 0: independent uniform like-probabilities (mean 1/2, no trend in
    the partner index); lambda = 0.75: everyone prefers the low-index users.
    The factors reproduce the preference matrices to their rank-d error."""
    mk0, P0, Q0 = crowding_market(200, 100, lam=0.0, d=16, seed=3)
    mk1, P1, Q1 = crowding_market(200, 100, lam=0.75, d=16, seed=3)
    assert P0.shape == (200, 100) and Q0.shape == (100, 200)
    assert abs(P0.mean() - 0.5) < 0.01 and abs(Q0.mean() - 0.5) < 0.01
    trend0 = np.corrcoef(np.arange(100), P0.mean(axis=0))[0, 1]
    trend1 = np.corrcoef(np.arange(100), P1.mean(axis=0))[0, 1]
    assert abs(trend0) < 0.3 and trend1 < -0.99
    for mk, P, Q in ((mk0, P0, Q0), (mk1, P1, Q1)):
        s = np.linalg.svd(P, compute_uv=False)
        err = np.linalg.norm(mk.F.astype(np.float64) @ mk.G.T.astype(np.float64) - P)
        assert err <= np.sqrt(np.sum(s[16:] ** 2)) * (1 + 1e-4)
        errq = np.linalg.norm(mk.K.astype(np.float64) @ mk.L.T.astype(np.float64) - Q.T)
        sq = np.linalg.svd(Q, compute_uv=False)
        assert errq <= np.sqrt(np.sum(sq[16:] ** 2)) * (1 + 1e-4)
