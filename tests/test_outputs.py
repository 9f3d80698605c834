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
        # sub-blocks into a host buffer with a leading dimension larger than
        # the width, at aligned and unaligned column offsets
        ld = 300
        for y0 in (1000, 1001, 3):
            out = np.full((40, ld), -1.0, np.float32)
            tu.tu_mu_block(mkt.handle, 100, 40, y0, 257, out, ld)
            np.testing.assert_allclose(out[:, :257], ref[100:140, y0:y0 + 257], rtol=EPS[path])
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
        # k <= 14: lists in shared memory; larger k: per-thread lists in local memory
        for k in (1, 10, 14, 15, 64):
            idx, lm = (t.cpu().numpy() for t in mkt.topk(side, k))
            _check_ranked(idx, lm.astype(np.float64), scores, EPS[path])
        # a row range into host buffers
        idx = np.empty((7, 10), np.int32)
        lmh = np.empty((7, 10), np.float32)
        tu.tu_topk_partners(mkt.handle, side, 10, 3, 7, idx, lmh)
        _check_ranked(idx, lmh.astype(np.float64), scores[3:10], EPS[path])
    finally:
        mkt.close()


@pytest.mark.parametrize("M,k", [(14, 14), (15, 14), (70, 14), (20, 20), (130, 20)])
def test_topk_k_near_partner_count(gpu_lib, M, k):
    """k up to the partner count: a column half of the one partner tile may
    hold fewer than k partners (its list stays padded) and the padded columns
    of the tile must never be listed."""
    tu = gpu_lib
    mk = make_market(300, M, 8, sigma=0.5, seed=11 + M, bias_x=True, bias_y=True, dtype="bf16")
    mkt = tu.from_synth(mk, path="fused")
    try:
        mkt.sweep(3)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        logA, _ = dense_logA(mk)
        scores = oracle.log_mu(logA, lu, lv)
        idx, lm = (t.cpu().numpy() for t in mkt.topk(0, k))
        assert idx.min() >= 0 and idx.max() < M
        _check_ranked(idx, lm.astype(np.float64), scores, EPS["fused"])
    finally:
        mkt.close()


@pytest.mark.parametrize("k", [14, 20])
def test_topk_ties_prefer_lower_index(gpu_lib, k):
    """Exactly tied partners (duplicated factor rows, no biases) are listed in
    increasing index order, whether the pair shares a column half of a partner
    tile or not (both list kinds: k = 14 and k = 20)."""
    tu = gpu_lib
    mk = make_market(40, 300, 8, sigma=1.0, seed=3, dtype="bf16")
    mk.G[150:] = mk.G[:150]
    mk.L[150:] = mk.L[:150]
    mkt = tu.from_synth(mk, path="fused")
    try:
        idx, _ = (t.cpu().numpy() for t in mkt.topk(0, k))
        for r in range(idx.shape[0]):
            for i in range(0, k, 2):
                a, b = idx[r, i], idx[r, i + 1]
                assert b == a + 150 and a < 150, (r, idx[r])
    finally:
        mkt.close()


def test_fused_topk_and_mu_full_size_sampled(gpu_lib):
    """1e6 x 1e6, d = 64 (the benchmark market) after one sweep: ranked lists of
    64 consecutive X users and 64 Y users over all 1e6 partners, and a mu block,
    against the oracle's log mu of those users computed from the GPU's potentials."""
    from synth import fused_market
    tu = gpu_lib
    mk = fused_market()
    stream = torch.cuda.Stream()
    mkt = tu.from_synth(mk, path="fused", stream=stream)
    try:
        mkt.sweep(1)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        f = mk.f64()
        s2 = 2.0 * f["sigma"]
        for side, row0 in ((0, 123457), (1, 876543)):
            if side == 0:
                A, B, own_b, par_b, lo, lp = mk.F, mk.K, mk.bias_x, mk.bias_y, lu, lv
                P, Q = mk.G, mk.L
            else:
                A, B, own_b, par_b, lo, lp = mk.G, mk.L, mk.bias_y, mk.bias_x, lv, lu
                P, Q = mk.F, mk.K
            rows = np.arange(row0, row0 + 64)
            phi = (A[rows].astype(np.float64) @ P.T.astype(np.float64)
                   + B[rows].astype(np.float64) @ Q.T.astype(np.float64)
                   + own_b[rows].astype(np.float64)[:, None] + par_b.astype(np.float64)[None, :])
            scores = phi / s2 + lo[rows][:, None] + lp[None, :]
            idx = torch.empty((64, 10), dtype=torch.int32, device="cuda")
            lm = torch.empty((64, 10), dtype=torch.float32, device="cuda")
            tu.tu_topk_partners(mkt.handle, side, 10, row0, 64, idx, lm)
            stream.synchronize()
            _check_ranked(idx.cpu().numpy(), lm.cpu().numpy().astype(np.float64), scores, EPS["fused"])
        # mu block at an unaligned partner offset, from potentials that put mu
        # near 1e-6 (one sweep from u = v = 1 leaves mu below the FP32 range)
        lu_set = (-7.0 - mk.bias_x.astype(np.float64) / s2).astype(np.float32)
        lv_set = (-7.0 - mk.bias_y.astype(np.float64) / s2).astype(np.float32)
        mkt.set_potentials(torch.from_numpy(lu_set).cuda(), torch.from_numpy(lv_set).cuda())
        rows = np.arange(123457, 123457 + 64)
        cols = slice(654321, 654321 + 5000)
        phi = (mk.F[rows].astype(np.float64) @ mk.G[cols].T.astype(np.float64)
               + mk.K[rows].astype(np.float64) @ mk.L[cols].T.astype(np.float64)
               + mk.bias_x[rows].astype(np.float64)[:, None] + mk.bias_y[cols].astype(np.float64)[None, :])
        ref = phi / s2 + lu_set[rows].astype(np.float64)[:, None] + lv_set[cols].astype(np.float64)[None, :]
        blk = torch.empty((64, 5000), dtype=torch.float32, device="cuda")
        tu.tu_mu_block(mkt.handle, 123457, 64, 654321, 5000, blk, 5000)
        stream.synchronize()
        got = blk.double().cpu().numpy()
        assert np.all(got > 0)
        np.testing.assert_allclose(np.log(got), ref, rtol=0, atol=3e-5)
    finally:
        mkt.close()


@pytest.mark.parametrize("path", ["fused", "dense"])
def test_topk_into_host_buffers_larger_than_the_staging(gpu_lib, path):
    """Ranked lists into host buffers whose two outputs together exceed the
    market's staging buffer as its creation left it (513 x 257, d = 8, k = 10:
    41 KB of outputs, 33 KB of staged factors): both views are taken from one
    staging buffer sized for both, and the lists equal those written into
    device buffers."""
    tu = gpu_lib
    mk = make_market(513, 257, 8, sigma=0.5, seed=5, bias_x=True, bias_y=True, n_kind="uniform1to3",
                     m_kind="uniform1to3", dtype="fp32")
    F, K, G, L = (np.ascontiguousarray(a, np.float32) for a in (mk.F, mk.K, mk.G, mk.L))
    h = tu.tu_market_create(F, K, G, L, mk.n, mk.m, mk.sigma, bias_x=mk.bias_x, bias_y=mk.bias_y, path=path)
    try:
        tu.tu_ipfp_sweep(h, 5)
        for side, rows in ((0, mk.N), (1, mk.M)):
            idx_h = np.empty((rows, 10), np.int32)
            lm_h = np.empty((rows, 10), np.float32)
            tu.tu_topk_partners(h, side, 10, 0, rows, idx_h, lm_h)
            idx_d = torch.empty((rows, 10), dtype=torch.int32, device="cuda")
            lm_d = torch.empty((rows, 10), dtype=torch.float32, device="cuda")
            tu.tu_topk_partners(h, side, 10, 0, rows, idx_d, lm_d)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(idx_h, idx_d.cpu().numpy())
            np.testing.assert_array_equal(lm_h, lm_d.cpu().numpy())
    finally:
        tu.tu_market_destroy(h)
