"""GPU parity of FP8 (e4m3) markets against the FP64 oracle run on the same
quantized factors (synth.fp8_quantized: the oracle side's own e4m3 rounding
and per-side power-of-two scale; the CUDA path quantizes with its own
conversion kernel).

The tensor cores multiply e4m3 values exactly and accumulate in FP32, so the
kernel's error budget is that of the BF16 path (ATOL_LOG, derived in
test_parity_fused.py); quantization itself is not an error here because the
oracle sees the same values. A single factor quantized differently moves phi
by about 2^-4 of one product, far above these tolerances."""

import numpy as np
import pytest
import torch

import oracle
from synth import fp8_quantized, fused_market, make_market

from _parity import oracle_solve, oracle_sweeps

pytestmark = pytest.mark.gpu

ATOL_LOG = 2e-5
MU_RTOL = 1e-3
MATCH_RTOL = 1e-5


def _mk(N, M, d, seed, **kw):
    base = dict(sigma=0.5, bias_x=True, bias_y=True, n_kind="uniform_real", m_kind="uniform_real", dtype="fp32")
    base.update(kw)
    return make_market(N, M, d, seed=seed, **base)


def test_fp8_phi_matches_quantized_factors(gpu_lib):
    """With u = v = 1, log mu = phi / (2 sigma): every pair checks the quantized
    inner product (and that the market is not computing with BF16 factors)."""
    tu = gpu_lib
    mk = _mk(700, 555, 64, seed=5, bias_x=False, bias_y=False)
    q, _ = fp8_quantized(mk)
    mkt = tu.from_synth(mk, fp8=True)
    try:
        lu = torch.zeros(mk.N, dtype=torch.float32, device="cuda")
        lv = torch.zeros(mk.M, dtype=torch.float32, device="cuda")
        mkt.set_potentials(lu, lv)
        got = torch.log(mkt.mu_block().double()).cpu().numpy()
        f = q.f64()
        want = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], None, None) / (2 * mk.sigma)
        np.testing.assert_allclose(got, want, rtol=0, atol=2e-6)
        fb = mk.f64()
        bf = oracle.phi_dense(fb["F"], fb["K"], fb["G"], fb["L"], None, None) / (2 * mk.sigma)
        assert np.abs(got - bf).max() > 1e-3  # FP8, not the unquantized product
    finally:
        mkt.close()


@pytest.mark.parametrize("N,M,d", [(700, 555, 64), (256, 128, 64), (333, 1201, 50), (1, 300, 24), (300, 1, 24),
                                   (1000, 1000, 16)], ids=lambda v: str(v))
def test_fp8_sweeps_match_oracle(gpu_lib, N, M, d):
    tu = gpu_lib
    mk = _mk(N, M, d, seed=N + 3 * M)
    q, _ = fp8_quantized(mk)
    mkt = tu.from_synth(mk, fp8=True)
    try:
        for target in (1, 4):
            mkt.sweep(target if target == 1 else target - 1)
            lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
            ou, ov = oracle_sweeps(q, target)
            np.testing.assert_allclose(lu, ou, rtol=0, atol=ATOL_LOG, err_msg=f"log u after {target}")
            np.testing.assert_allclose(lv, ov, rtol=0, atol=ATOL_LOG, err_msg=f"log v after {target}")
    finally:
        mkt.close()


def test_fp8_solve_and_ranked_lists(gpu_lib):
    tu = gpu_lib
    mk = _mk(900, 1400, 64, seed=11)
    q, _ = fp8_quantized(mk)
    mkt = tu.from_synth(mk, fp8=True)
    try:
        info = mkt.solve(tol=1e-6, max_iter=5000)
        assert info["converged"], info
        r, logA, f = oracle_solve(q)
        mu_ref = np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))
        np.testing.assert_allclose(mkt.mu_block().double().cpu().numpy(), mu_ref, rtol=MU_RTOL, atol=0)
        cx = oracle.match_count(f["n"], r["log_u"])
        assert abs(info["match_count"] - cx) <= MATCH_RTOL * cx
        idx, lm = mkt.topk(0, 10)
        lmu = oracle.log_mu(logA, r["log_u"], r["log_v"])
        want = np.argsort(-lmu, axis=1, kind="stable")[:, :10]
        got = idx.cpu().numpy()
        # ranks agree wherever the oracle's neighbouring scores are separated
        srt = -np.sort(-lmu, axis=1)[:, :11]
        clear = (srt[:, :10] - srt[:, 1:11]) > 1e-4
        clear[:, 1:] &= (srt[:, :9] - srt[:, 1:10]) > 1e-4
        assert np.all(got[clear] == want[clear])
        np.testing.assert_allclose(lm.double().cpu().numpy(), np.take_along_axis(lmu, got.astype(np.int64), 1),
                                   rtol=0, atol=1e-4)
    finally:
        mkt.close()


def test_fp8_batch_bit_identical_to_solo(gpu_lib):
    tu = gpu_lib
    shapes = [(700, 555, 64), (300, 1000, 48), (1, 300, 24), (513, 257, 64)]
    mks = [_mk(N, M, d, seed=50 + i) for i, (N, M, d) in enumerate(shapes)]
    solo = [tu.from_synth(mk, fp8=True) for mk in mks]
    grouped = [tu.from_synth(mk, fp8=True) for mk in mks]
    batch = tu.Batch(grouped)
    try:
        batch.sweep(3)
        torch.cuda.synchronize()
        for m in solo:
            m.sweep(3)
        for a, b in zip(solo, grouped):
            (au, av), (bu, bv) = a.potentials(), b.potentials()
            assert torch.equal(au, bu) and torch.equal(av, bv)
    finally:
        batch.close()
        for m in solo + grouped:
            m.close()


def test_fp8_invalid_combinations(gpu_lib):
    tu = gpu_lib
    mk = _mk(100, 120, 32, seed=3)
    with pytest.raises(tu.TuError) as e:
        tu.from_synth(mk, path="dense", fp8=True)
    assert e.value.status == tu.TU_ERR_UNSUPPORTED
    a = tu.from_synth(mk, fp8=True)
    b = tu.from_synth(_mk(100, 120, 64, seed=4, dtype="bf16"))
    try:
        with pytest.raises(tu.TuError) as e:
            tu.tu_batch_create([a.handle, b.handle])
        assert e.value.status == tu.TU_ERR_INVALID_ARG
    finally:
        a.close()
        b.close()


def test_fp8_full_size_sampled_sweep(gpu_lib):
    """The 1e6 x 1e6 workload (d = 64, lognormal biases) with FP8 factors: one
    sweep, sampled users of both sides against the oracle's mini-batch update
    on the quantized factors."""
    tu = gpu_lib
    mk = fused_market(dtype="fp32")
    q, _ = fp8_quantized(mk)
    mkt = tu.from_synth(mk, fp8=True)
    rng = np.random.default_rng(9)
    try:
        mkt.set_translation(False)  # one sweep of Eq. iteration
        mkt.sweep(1)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        f = q.f64()
        rows = rng.choice(mk.N, 64, replace=False)
        cols = rng.choice(mk.M, 64, replace=False)
        _, ou = oracle.sampled_row_update(q.F, q.K, q.G, q.L, f["sigma"], f["n"], np.zeros(mk.M), rows,
                                          q.bias_x, q.bias_y)
        _, ov = oracle.sampled_row_update(q.G, q.L, q.F, q.K, f["sigma"], f["m"], lu, cols, q.bias_y, q.bias_x)
        np.testing.assert_allclose(lu[rows], ou, rtol=0, atol=ATOL_LOG)
        np.testing.assert_allclose(lv[cols], ov, rtol=0, atol=ATOL_LOG)
    finally:
        mkt.close()
