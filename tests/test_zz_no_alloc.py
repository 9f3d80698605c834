"""The allocation-free half-sweep entry point against the market path.

tu_fused_halfsweep_noalloc serves callers that cannot call cudaMalloc (device
memory fully budgeted by an admission controller or held by another
allocator; latency-critical loops where an allocation would synchronise the
device). Its scratch is a fixed file-scope device array shared by all calls,
so this test calls it twice in a row and checks both results against the u
step of an ordinary market sweep (tu_ipfp_sweep) from the same state, with
the tolerance the fused parity tests use. This file is named so that pytest
collects it last.
"""

import numpy as np
import pytest
import torch

from synth import make_market

pytestmark = pytest.mark.gpu

ATOL_LOG = 2e-5  # same bound as the fused parity tests


def _packed(A, B, kp):
    rows, d = A.shape
    out = np.zeros((rows, kp), np.float32)
    out[:, :d] = A
    out[:, d:2 * d] = B
    bits = (out.view(np.uint32) >> 16).astype(np.uint16)
    return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()


@pytest.mark.parametrize("N,M,d,kp", [(700, 555, 64, 128), (4099, 3001, 24, 64)])
def test_noalloc_matches_market_half_sweep_twice(gpu_lib, N, M, d, kp):
    tu = gpu_lib
    mk = make_market(N, M, d, sigma=0.5, seed=N + M, bias_x=True, bias_y=True, n_kind="uniform_real",
                     m_kind="uniform_real", dtype="bf16")
    rng = np.random.default_rng(3)
    lu0 = rng.normal(-3.0, 0.5, N).astype(np.float32)
    lv0 = rng.normal(-3.0, 0.5, M).astype(np.float32)
    lu0_t, lv0_t = torch.from_numpy(lu0).cuda(), torch.from_numpy(lv0).cuda()

    # existing entry points: residual of the state, then the u step of one sweep
    mkt = tu.from_synth(mk, path="fused")
    try:
        mkt.set_translation(False)  # the u step of Eq. iteration, as the entry point computes
        mkt.set_potentials(lu0_t, lv0_t)
        res_market = tu.tu_ipfp_sweep(mkt.handle, 0, residual=True)
        mkt.sweep(1)
        lu_market = mkt.potentials()[0].cpu().numpy()
    finally:
        mkt.close()

    own = _packed(mk.F, mk.K, kp)
    par = _packed(mk.G, mk.L, kp)
    bx = torch.from_numpy(mk.bias_x).cuda()
    by = torch.from_numpy(mk.bias_y).cuda()
    mass = torch.from_numpy(mk.n).cuda()
    torch.cuda.synchronize()
    outs = []
    for _ in range(2):
        out = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
        res = tu.tu_fused_halfsweep_noalloc(N, M, kp, own, par, bx, mass, lu0_t, by, lv0_t, mk.sigma, out,
                                            residual=True)
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, lu_market, rtol=0, atol=ATOL_LOG)
        assert abs(res - res_market) <= 1e-5 * max(1.0, res_market)
        outs.append(got)
    np.testing.assert_array_equal(outs[0], outs[1])


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu_lib):
    tu = gpu_lib
    t = torch.zeros(128, dtype=torch.float32, device="cuda")
    p = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    m = torch.ones(128, dtype=torch.float64, device="cuda")
    for rows, cols, kp in [(65537, 10, 64), (10, (1 << 20) + 1, 64), (10, 10, 192)]:
        with pytest.raises(tu.TuError) as e:
            tu.tu_fused_halfsweep_noalloc(rows, cols, kp, p, p, None, m, t, None, t, 0.5, t)
        assert e.value.status == tu.TU_ERR_UNSUPPORTED
    # host memory is refused (the entry point never stages through a copy)
    h = np.zeros(128, np.float32)
    with pytest.raises(tu.TuError) as e:
        tu.tu_fused_halfsweep_noalloc(10, 10, 64, p, p, None, m, h, None, t, 0.5, t)
    assert e.value.status == tu.TU_ERR_INVALID_ARG


def test_noalloc_reports_nonfinite_potentials_when_asked(gpu_lib):
    """A NaN among the partner potentials makes computed potentials NaN: with
    residual_out the call synchronises and returns TU_ERR_NONFINITE; without it
    the call only enqueues work and reports nothing (the header says so). The
    device check of every pointer (a buffer of another device or host memory
    is refused) is exercised by the host-pointer case of the refusal test; a
    second GPU is not available here."""
    tu = gpu_lib
    N, M, d, kp = 300, 257, 16, 64
    mk = make_market(N, M, d, sigma=0.5, seed=5, dtype="bf16")
    own = _packed(mk.F, mk.K, kp)
    par = _packed(mk.G, mk.L, kp)
    mass = torch.from_numpy(mk.n).cuda()
    lu0 = torch.zeros(N, dtype=torch.float32, device="cuda")
    lv0 = torch.zeros(M, dtype=torch.float32, device="cuda")
    lv0[17] = float("nan")
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    tu.tu_fused_halfsweep_noalloc(N, M, kp, own, par, None, mass, lu0, None, lv0, mk.sigma, out)
    torch.cuda.synchronize()
    with pytest.raises(tu.TuError) as e:
        tu.tu_fused_halfsweep_noalloc(N, M, kp, own, par, None, mass, lu0, None, lv0, mk.sigma, out, residual=True)
    assert e.value.status == tu.TU_ERR_NONFINITE
    # the shared scratch is usable again by the next call
    lv0[17] = 0.0
    res = tu.tu_fused_halfsweep_noalloc(N, M, kp, own, par, None, mass, lu0, None, lv0, mk.sigma, out,
                                        residual=True)
    assert np.isfinite(res) and torch.isfinite(out).all()
