"""GPU parity of the output stage: blocks of mu and ranked partner lists.

Ranked lists: indices must equal the oracle's wherever the oracle's score gap
to both neighbours exceeds EPS (a bound on the GPU score error); inside a gap
below EPS either order is correct, so there the chosen partner's oracle score
must lie within EPS of the oracle's score at that rank.
"""

import numpy as np
import pytest
import torch

import oracle
from synth import make_market

from _parity import dense_logA

pytestmark = pytest.mark.gpu

# log mu is returned in FP32: at |log mu| ~ 16 one FP32 spacing is 1.9e-6 and the
# score is the sum of three rounded terms, so the dense path is held to 1e-5;
# the fused path adds the BF16-product / FP32-accumulation error of phi (2e-5).
EPS = {"fused": 2e-5, "dense": 1e-5}


def _market(path, N=517, M=1333, d=32, seed=21):
    dtype = "bf16" if path == "fused" else "fp32"
    return make_market(N, M, d, sigma=0.5, seed=seed, bias_x=True, bias_y=True, n_kind="uniform_real",
                       m_kind="uniform1to3", dtype=dtype)


def _check_ranked(idx, lm_gpu, scores, eps):
    """idx, lm_gpu: GPU lists (rows x k); scores: oracle log mu (rows x partners)."""
    k = idx.shape[1]
    order = np.argsort(-scores, axis=1, kind="stable")
    for r in range(idx.shape[0]):
        s_sorted = scores[r, order[r]]
        assert len(set(idx[r].tolist())) == k
        for i in range(k):
            gap_lo = s_sorted[i - 1] - s_sorted[i] if i > 0 else np.inf
            gap_hi = s_sorted[i] - s_sorted[i + 1] if i + 1 < len(s_sorted) else np.inf
            if min(gap_lo, gap_hi) > eps:
                assert idx[r, i] == order[r, i], (r, i)
            else:
                assert abs(scores[r, idx[r, i]] - s_sorted[i]) <= eps, (r, i)
            assert abs(lm_gpu[r, i] - scores[r, idx[r, i]]) <= eps


@pytest.mark.parametrize("path", ["fused", "dense"])
def test_mu_block_matches_oracle(gpu_lib, path):
    tu = gpu_lib
    mk = _market(path)
    mkt = tu.from_synth(mk, path=path)
    try:
        mkt.sweep(5)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        logA, _ = dense_logA(mk)
        ref = np.exp(oracle.log_mu(logA, lu, lv))
        full = mkt.mu_block().double().cpu().numpy()
        np.testing.assert_allclose(full, ref, rtol=EPS[path])
        # a sub-block into a host buffer with a leading dimension larger than its width
        ld = 300
        out = np.full((40, ld), -1.0, np.float32)
        tu.tu_mu_block(mkt.handle, 100, 40, 1000, 257, out, ld)
        np.testing.assert_allclose(out[:, :257], ref[100:140, 1000:1257], rtol=EPS[path])
        assert np.all(out[:, 257:] == -1.0)
    finally:
        mkt.close()


@pytest.mark.parametrize("path", ["fused", "dense"])
@pytest.mark.parametrize("side", [0, 1])
def test_topk_matches_oracle(gpu_lib, path, side):
    tu = gpu_lib
    mk = _market(path)
    mkt = tu.from_synth(mk, path=path)
    try:
        mkt.sweep(5)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        logA, _ = dense_logA(mk)
        scores = oracle.log_mu(logA, lu, lv)
        if side == 1:
            scores = scores.T
        for k in (1, 10, 64):
            idx, lm = (t.cpu().numpy() for t in mkt.topk(side, k))
            _check_ranked(idx, lm.astype(np.float64), scores, EPS[path])
        # a row range into host buffers
        idx = np.empty((7, 10), np.int32)
        lmh = np.empty((7, 10), np.float32)
        tu.tu_topk_partners(mkt.handle, side, 10, 3, 7, idx, lmh)
        _check_ranked(idx, lmh.astype(np.float64), scores[3:10], EPS[path])
    finally:
        mkt.close()


def test_topk_ties_prefer_lower_index(gpu_lib):
    """Exactly tied partners (duplicated factor rows, no biases) are listed in
    increasing index order."""
    tu = gpu_lib
    mk = make_market(40, 300, 8, sigma=1.0, seed=3, dtype="bf16")
    mk.G[150:] = mk.G[:150]
    mk.L[150:] = mk.L[:150]
    mkt = tu.from_synth(mk, path="fused")
    try:
        idx, _ = (t.cpu().numpy() for t in mkt.topk(0, 20))
        for r in range(idx.shape[0]):
            for i in range(0, 20, 2):
                a, b = idx[r, i], idx[r, i + 1]
                assert b == a + 150 and a < 150, (r, idx[r])
    finally:
        mkt.close()
