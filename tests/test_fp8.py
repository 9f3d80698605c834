"""GPU parity of FP8 (e4m3) markets against the FP64 oracle run on the same
quantized factors (synth.fp8_quantized: the oracle side's own e4m3 rounding
and per-row power-of-two scales; the CUDA path quantizes with its own
conversion kernel, or takes the caller's bytes and scales).

The tensor cores multiply e4m3 values exactly and accumulate in FP32, so the
kernel's error budget is that of the BF16 path (ATOL_LOG, derived in
test_parity_fused.py); quantization itself is not an error here because the
oracle sees the same values. A single factor quantized differently moves phi
by about 2^-4 of one product, far above these tolerances."""

import numpy as np
import pytest
import torch

import oracle
from synth import fp8_encoded, fp8_quantized, fused_market, make_market

from _parity import oracle_solve, oracle_sweeps

pytestmark = pytest.mark.gpu

ATOL_LOG = 2e-5
MU_RTOL = 1e-3
MATCH_RTOL = 1e-5


def _mk(N, M, d, seed, **kw):
    base = dict(sigma=0.5, bias_x=True, bias_y=True, n_kind="uniform_real", m_kind="uniform_real", dtype="fp32")
    base.update(kw)
    return make_market(N, M, d, seed=seed, **base)


@pytest.mark.parametrize("per", ["row", "side"])
def test_fp8_phi_matches_quantized_factors(gpu_lib, per):
    """With u = v = 1, log mu = phi / (2 sigma): every pair checks the quantized
    inner product (and that the market is not computing with BF16 factors),
    with per-row and per-side scales."""
    tu = gpu_lib
    mk = _mk(700, 555, 64, seed=5, bias_x=False, bias_y=False)
    q, _ = fp8_quantized(mk, per)
    mkt = tu.from_synth(mk, fp8="rows" if per == "row" else "side")
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


# d = 65..128: packed rows of two 128-byte k blocks; d = 129..256: four
@pytest.mark.parametrize("N,M,d,per", [(700, 555, 64, "row"), (256, 128, 64, "row"), (333, 1201, 50, "row"),
                                       (1, 300, 24, "row"), (300, 1, 24, "row"), (1000, 1000, 16, "row"),
                                       (700, 555, 128, "row"), (257, 129, 65, "row"), (300, 700, 200, "row"),
                                       (700, 555, 64, "side"), (1, 300, 24, "side"), (300, 700, 200, "side")],
                         ids=lambda v: str(v))
def test_fp8_sweeps_match_oracle(gpu_lib, N, M, d, per):
    tu = gpu_lib
    mk = _mk(N, M, d, seed=N + 3 * M)
    q, _ = fp8_quantized(mk, per)
    mkt = tu.from_synth(mk, fp8="rows" if per == "row" else "side")
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


@pytest.mark.parametrize("mode", ["rows", "side"])
def test_fp8_batch_bit_identical_to_solo(gpu_lib, mode):
    tu = gpu_lib
    shapes = [(700, 555, 64), (300, 1000, 48), (1, 300, 24), (513, 257, 64)]
    mks = [_mk(N, M, d, seed=50 + i) for i, (N, M, d) in enumerate(shapes)]
    solo = [tu.from_synth(mk, fp8=mode) for mk in mks]
    grouped = [tu.from_synth(mk, fp8=mode) for mk in mks]
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


def test_batch_follows_replaced_factors(gpu_lib):
    """A batch holds its members' descriptors, built at creation. Replacing a
    member's factors moves an e4m3 market's side scales and with them the
    exponent multiplier c = log2(e) / (2 sigma) 2^(k_X + k_Y), which the
    batch must follow: after the same replacement, batched sweeps stay bit
    for bit those of the market alone. Factors that become wide are refused
    at the next batch call (TU_ERR_UNSUPPORTED), and accepted again once
    replaced by narrow ones."""
    tu = gpu_lib
    mks = [_mk(400, 300, 64, seed=70), _mk(300, 500, 48, seed=71)]
    solo = [tu.from_synth(mk, fp8="side") for mk in mks]
    grouped = [tu.from_synth(mk, fp8="side") for mk in mks]
    batch = tu.Batch(grouped)

    def cuda(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()

    def same():
        for a, b in zip(solo, grouped):
            (au, av), (bu, bv) = a.potentials(), b.potentials()
            assert torch.equal(au, bu) and torch.equal(av, bv)

    try:
        batch.sweep(2)
        torch.cuda.synchronize()
        for m in solo:
            m.sweep(2)
        same()
        # 8 x the X factors of market 0: its X scale exponent moves by 3
        mk = mks[0]
        new = (cuda(8.0 * mk.F), cuda(8.0 * mk.K), cuda(mk.G), cuda(mk.L))
        for m in (solo[0], grouped[0]):
            m.update_factors(*new)
        batch.sweep(2)
        torch.cuda.synchronize()
        for m in solo:
            m.sweep(2)
        same()
        # 40 x: beyond one shift per half-sweep
        wide = (cuda(40.0 * mk.F), cuda(40.0 * mk.K), cuda(40.0 * mk.G), cuda(40.0 * mk.L))
        grouped[0].update_factors(*wide)
        with pytest.raises(tu.TuError) as e:
            batch.sweep(1)
        assert e.value.status == tu.TU_ERR_UNSUPPORTED
        grouped[0].update_factors(*new)
        batch.sweep(1)
        torch.cuda.synchronize()
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
    # the batched kernel takes BF16 rows of up to two k blocks (d <= 64) and e4m3 rows of one
    c = tu.from_synth(_mk(100, 120, 100, seed=5, dtype="bf16"))
    f = tu.from_synth(_mk(100, 120, 100, seed=6), fp8=True)
    s = tu.from_synth(_mk(100, 120, 32, seed=7), fp8="side")
    try:
        for other in (b, s):  # one operand format per batch
            with pytest.raises(tu.TuError) as e:
                tu.tu_batch_create([a.handle, other.handle])
            assert e.value.status == tu.TU_ERR_INVALID_ARG
        for h in (c.handle, f.handle):
            with pytest.raises(tu.TuError) as e:
                tu.tu_batch_create([h])
            assert e.value.status == tu.TU_ERR_UNSUPPORTED
    finally:
        for m in (a, b, c, f, s):
            m.close()


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


def _scaled_rows(mk, fx=1e-4, fy=1e-3):
    """The market with every other X row and every third Y row scaled down
    (factors of very different norms within a side)."""
    import dataclasses
    sx = np.where(np.arange(mk.N) % 2 == 0, fx, 1.0).astype(np.float32)[:, None]
    sy = np.where(np.arange(mk.M) % 3 == 0, fy, 1.0).astype(np.float32)[:, None]
    return dataclasses.replace(mk, F=mk.F * sx, K=mk.K * sx, G=mk.G * sy, L=mk.L * sy)


def test_fp8_row_scales_with_rows_of_different_norms(gpu_lib):
    """Rows 1e-4 (X) and 1e-3 (Y) the size of the others: each row keeps its
    own scale, phi of every pair matches the quantized factors (u = v = 1),
    and the sweeps match the oracle."""
    tu = gpu_lib
    mk = _scaled_rows(_mk(640, 384, 64, seed=31, bias_x=False, bias_y=False))
    q, (kx, ky) = fp8_quantized(mk)
    assert kx.max() - kx.min() >= 12 and ky.max() - ky.min() >= 8  # the scales differ per row
    mkt = tu.from_synth(mk, fp8=True)
    try:
        mkt.set_potentials(torch.zeros(mk.N, dtype=torch.float32, device="cuda"),
                           torch.zeros(mk.M, dtype=torch.float32, device="cuda"))
        got = torch.log(mkt.mu_block().double()).cpu().numpy()
        f = q.f64()
        want = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], None, None) / (2 * mk.sigma)
        np.testing.assert_allclose(got, want, rtol=0, atol=2e-6 * max(1.0, np.abs(want).max()))
        mkt.sweep(3)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        ou, ov = oracle_sweeps(q, 3)
        np.testing.assert_allclose(lu, ou, rtol=0, atol=ATOL_LOG)
        np.testing.assert_allclose(lv, ov, rtol=0, atol=ATOL_LOG)
    finally:
        mkt.close()


def test_fp8_caller_scales_equal_library_quantization(gpu_lib):
    """A caller that quantizes the rows itself (e4m3 bytes and per-row FP32
    scales, synth.fp8_encoded; device or host buffers) gets the library's own
    quantization of the same FP32 factors bit for bit; the scaled update
    replaces them like a new market's."""
    tu = gpu_lib
    mk = _scaled_rows(_mk(700, 555, 100, seed=21))
    mk2 = _mk(700, 555, 100, seed=22)

    def cuda(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    enc = fp8_encoded(mk)
    lib_q = tu.from_synth(mk, fp8=True)
    bx, by = cuda(mk.bias_x), cuda(mk.bias_y)
    dev = tu.Market(*(cuda(a) for a in enc[:4]), mk.n, mk.m, mk.sigma, bias_x=bx, bias_y=by, fp8=True,
                    fscale_x=cuda(enc[4]), fscale_y=cuda(enc[5]))
    host = tu.Market(*enc[:4], mk.n, mk.m, mk.sigma, bias_x=bx, bias_y=by, fp8=True, fscale_x=enc[4],
                     fscale_y=enc[5])
    other = tu.from_synth(mk2, fp8=True)
    try:
        for m in (lib_q, dev, host):
            m.sweep(3)
        ref = lib_q.potentials()
        for m in (dev, host):
            got = m.potentials()
            assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
        # scaled update: the factors of mk2 (biases of mk stay), warm-started potentials kept
        enc2 = fp8_encoded(mk2)
        tu.tu_market_update_factors_fp8(dev.handle, *(cuda(a) for a in enc2))
        tu.tu_market_update_factors(lib_q.handle, *(torch.from_numpy(a).cuda() for a in (mk2.F, mk2.K, mk2.G,
                                                                                         mk2.L)))
        dev.sweep(2)
        lib_q.sweep(2)
        a, b = dev.potentials(), lib_q.potentials()
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
        # each market takes only its own kind of update
        with pytest.raises(tu.TuError) as e:
            tu.tu_market_update_factors(dev.handle, *(cuda(a) for a in enc2[:4]))
        assert e.value.status == tu.TU_ERR_INVALID_ARG
        with pytest.raises(tu.TuError) as e:
            tu.tu_market_update_factors_fp8(other.handle, *(cuda(a) for a in enc2))
        assert e.value.status == tu.TU_ERR_INVALID_ARG
        bad = enc2[4].copy()
        bad[5] = np.nan
        with pytest.raises(tu.TuError) as e:
            tu.tu_market_update_factors_fp8(dev.handle, *(cuda(a) for a in enc2[:4]), cuda(bad), cuda(enc2[5]))
        assert e.value.status == tu.TU_ERR_NONFINITE
    finally:
        for m in (lib_q, dev, host, other):
            m.close()
