"""Every documented error of the market entry points (GPU): the call returns
its status, and, since none of these is TU_ERR_CUDA, the market is not
poisoned: after the error the same market sweeps exactly like a market that
never saw it."""

import numpy as np
import pytest
import torch

from synth import make_market

pytestmark = pytest.mark.gpu


def _mk(seed=5, **kw):
    base = dict(sigma=0.5, bias_x=True, bias_y=True, n_kind="uniform1to3", m_kind="uniform1to3", dtype="bf16")
    base.update(kw)
    return make_market(300, 200, 16, seed=seed, **base)


def _factor(a, path):
    """A factor matrix in the market's element type (bf16 bit patterns on the fused path, float32 on the dense one)."""
    a = np.ascontiguousarray(a, np.float32)
    if path == "fused":
        bits = (a.view(np.uint32) >> 16).astype(np.uint16)
        return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(a).cuda()


def _status(fn, *a):
    import paper_2411_19214_gb300 as tu
    with pytest.raises(tu.TuError) as e:
        fn(*a)
    return e.value.status


def _still_sweeps_like_fresh(tu, mkt, mk, path="fused"):
    fresh = tu.from_synth(mk, path=path)
    try:
        lu, lv = fresh.potentials()
        mkt.set_potentials(lu, lv)
        fresh.sweep(2)
        mkt.sweep(2)
        for a, b in zip(mkt.potentials(), fresh.potentials()):
            assert torch.equal(a, b)
    finally:
        fresh.close()


@pytest.mark.parametrize("path", ["fused", "dense"])
def test_call_errors_leave_the_market_usable(gpu_lib, path):
    tu = gpu_lib
    mk = _mk(dtype="bf16" if path == "fused" else "fp32")
    mkt = tu.from_synth(mk, path=path)
    h = mkt.handle
    N, M = mk.N, mk.M
    idx = torch.empty((N, 70), dtype=torch.int32, device="cuda")
    lm = torch.empty((N, 70), dtype=torch.float32, device="cuda")
    out = torch.empty((N, M), dtype=torch.float32, device="cuda")
    try:
        INV = tu.TU_ERR_INVALID_ARG
        assert _status(tu.tu_ipfp_sweep, h, -1) == INV
        for side, k, row0, nrows in [(2, 10, 0, N), (0, 0, 0, N), (0, 65, 0, N), (1, M + 1, 0, 10),
                                     (0, 10, -1, 5), (0, 10, N - 4, 5), (1, 10, 0, M + 1), (0, 10, 0, -1)]:
            st = _status(tu.tu_topk_partners, h, side, k, row0, nrows, idx, lm)
            assert st == INV, (side, k, row0, nrows, st)
        for x0, nx, y0, ny, ld in [(-1, 5, 0, 5, 5), (0, N + 1, 0, 5, 5), (0, 5, M - 2, 5, 5), (0, 5, 0, 5, 4),
                                   (0, -1, 0, 5, 5)]:
            st = _status(tu.tu_mu_block, h, x0, nx, y0, ny, out, ld)
            assert st == INV, (x0, nx, y0, ny, ld, st)
        for omega in (-0.5, 0.5, 2.0, float("nan")):
            assert _status(tu.tu_market_set_relaxation, h, omega) == INV, omega
        assert _status(tu.tu_market_relax_update, h, -1.0) == INV
        for bad in (dict(k=0), dict(k=64), dict(sample=0), dict(check_every=0), dict(patience=0),
                    dict(score_eps=-1.0), dict(max_iter=-1)):
            kw = dict(k=5, sample=16, check_every=2, patience=2, max_iter=10)
            kw.update(bad)
            assert _status(lambda: mkt.solve_ranking(**kw)) == INV, bad
        # non-finite factors in an update: refused; the factors are undefined until
        # the next successful update, which restores the market
        Fn = mk.F.copy()
        Fn[3, 2] = np.nan
        facs = [_factor(a, path) for a in (Fn, mk.K, mk.G, mk.L)]
        assert _status(tu.tu_market_update_factors, h, *facs) == tu.TU_ERR_NONFINITE
        tu.tu_market_update_factors(h, *(_factor(a, path) for a in (mk.F, mk.K, mk.G, mk.L)))
        _still_sweeps_like_fresh(tu, mkt, mk, path)
    finally:
        mkt.close()


def test_nonfinite_potentials_are_reported_and_recoverable(gpu_lib):
    """A NaN in log v reaches every u of the next X half-sweep (u is
    recomputed from v, so a NaN in log u alone is simply overwritten): the
    sweep reports TU_ERR_NONFINITE, and restored potentials recover."""
    tu = gpu_lib
    mk = _mk(seed=6)
    mkt = tu.from_synth(mk)
    try:
        lu, lv = mkt.potentials()
        bad_u = lu.clone()
        bad_u[17] = float("nan")
        mkt.set_potentials(bad_u, lv)
        assert np.isfinite(tu.tu_ipfp_sweep(mkt.handle, 1, True))
        bad_v = lv.clone()
        bad_v[17] = float("nan")
        mkt.set_potentials(lu, bad_v)
        st = _status(tu.tu_ipfp_sweep, mkt.handle, 1, True)
        assert st == tu.TU_ERR_NONFINITE
        _still_sweeps_like_fresh(tu, mkt, mk)
    finally:
        mkt.close()


@pytest.mark.parametrize("path,fp8", [("fused", False), ("fused", True), ("dense", False)])
def test_nan_factors_refused(gpu_lib, path, fp8):
    """A NaN factor entry (not only an infinite one) is refused at creation and
    in an update, on every path."""
    tu = gpu_lib
    mk = _mk(seed=12, dtype="fp32")
    F = mk.F.copy()
    F[5, 1] = np.nan
    st = _status(lambda: tu.tu_market_create(F, mk.K, mk.G, mk.L, mk.n, mk.m, mk.sigma, path=path, fp8=fp8))
    assert st == tu.TU_ERR_NONFINITE
    mkt = tu.Market(mk.F, mk.K, mk.G, mk.L, mk.n, mk.m, mk.sigma, path=path, fp8=fp8)
    try:
        L = mk.L.copy()
        L[3, 0] = np.nan
        assert _status(tu.tu_market_update_factors, mkt.handle, mk.F, mk.K, mk.G, L) == tu.TU_ERR_NONFINITE
    finally:
        mkt.close()


def test_create_errors(gpu_lib):
    tu = gpu_lib
    mk = _mk(seed=7)
    for n, m in [(np.r_[mk.n[:-1], 0.0], mk.m), (mk.n, np.r_[mk.m[:-1], -1.0]), (np.r_[np.nan, mk.n[1:]], mk.m),
                 (mk.n, np.r_[np.inf, mk.m[1:]])]:
        st = _status(tu.tu_market_create, mk.F, mk.K, mk.G, mk.L, n, m, mk.sigma)
        assert st == tu.TU_ERR_INVALID_ARG
    F = mk.F.copy()
    F[0, 0] = np.inf
    assert _status(tu.tu_market_create, F, mk.K, mk.G, mk.L, mk.n, mk.m, mk.sigma) == tu.TU_ERR_NONFINITE
    for name, bad in (("bias_x", np.r_[mk.bias_x[:-1], np.nan]), ("bias_y", np.r_[np.inf, mk.bias_y[1:]])):
        kw = dict(bias_x=mk.bias_x, bias_y=mk.bias_y)
        kw[name] = bad.astype(np.float32)
        st = _status(lambda: tu.tu_market_create(mk.F, mk.K, mk.G, mk.L, mk.n, mk.m, mk.sigma, **kw))
        assert st == tu.TU_ERR_NONFINITE, name
    # max|a| max|b| / (2 sigma) far above 40: outside the FP32 range of the dense
    # path's A-hat (the fused path takes such markets with per-row shifts)
    big = make_market(300, 200, 16, sigma=0.5, seed=8, factor_scale=60.0, dtype="fp32")
    st = _status(lambda: tu.tu_market_create(big.F, big.K, big.G, big.L, big.n, big.m, big.sigma, path="dense"))
    assert st == tu.TU_ERR_UNSUPPORTED
