"""Host-side request validation of the serving loop (no GPU): a malformed
request is answered `invalid` before it is admitted, with the reason."""

import numpy as np
import pytest

from synth import make_market


def _req(serve, **over):
    mk = make_market(30, 40, 8, sigma=0.5, seed=1, bias_x=True, bias_y=True, n_kind="uniform1to3",
                     m_kind="uniform1to3", dtype="bf16")
    kw = dict(rid=0, arrival=0.0, F=mk.F, K=mk.K, G=mk.G, L=mk.L, n=mk.n, m=mk.m, sigma=mk.sigma,
              bias_x=mk.bias_x, bias_y=mk.bias_y)
    kw.update(over)
    return serve.SolveRequest(**kw)


def test_valid_request_passes():
    from paper_2411_19214_gb300 import serve
    assert serve.validate(_req(serve)) is None
    # sigma as any real scalar: Python int or numpy float32 / float64
    for sigma in (1, np.float32(0.5), np.float64(0.25)):
        assert serve.validate(_req(serve, sigma=sigma)) is None, sigma


@pytest.mark.parametrize("over,needle", [
    (dict(K=np.zeros((30, 7), np.float32)), "share one"),
    (dict(L=np.zeros((41, 8), np.float32)), "share one"),
    (dict(G=np.zeros((40, 9), np.float32), L=np.zeros((40, 9), np.float32)), "same d"),
    (dict(F=np.zeros((30, 129), np.float32), K=np.zeros((30, 129), np.float32),
          G=np.zeros((40, 129), np.float32), L=np.zeros((40, 129), np.float32)), "limit"),
    (dict(n=np.ones(29)), "one capacity per user"),
    (dict(m=np.r_[np.ones(39), 0.0]), "finite and > 0"),
    (dict(n=np.r_[np.ones(29), np.nan]), "finite and > 0"),
    (dict(m=-np.ones(40)), "finite and > 0"),
    (dict(sigma=0.0), "sigma"),
    (dict(sigma=float("inf")), "sigma"),
    (dict(sigma=np.float32("nan")), "sigma"),
    (dict(sigma=True), "sigma"),
    (dict(sigma="0.5"), "sigma"),
    (dict(sigma=np.array([0.5])), "sigma"),
    (dict(bias_x=np.zeros(31, np.float32)), "bias_x"),
    (dict(bias_y=np.zeros((40, 1), np.float32)), "bias_y"),
])
def test_malformed_requests_are_named(over, needle):
    from paper_2411_19214_gb300 import serve
    why = serve.validate(_req(serve, **over))
    assert why is not None and needle in why, why


class _FakeLib:
    """The library calls of the micro-batching server, faked on the host: markets
    are integers, a batch refuses every group (as it refuses a group holding a
    market with a wide exponent range), single-market solves succeed except
    for the handles listed in `fail`."""

    def __init__(self, serve, monkeypatch, fail=()):
        import torch
        self.created, self.destroyed, self.solved, self.fail = [], [], [], set(fail)
        self.TuError = serve.TuError
        monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
        for name in ("tu_market_footprint", "tu_market_create", "tu_market_destroy", "tu_market_set_translation",
                     "tu_market_set_relaxation", "tu_batch_create", "tu_batch_destroy", "tu_batch_solve",
                     "tu_ipfp_solve", "tu_topk_partners", "tu_market_update_factors"):
            monkeypatch.setattr(serve, name, getattr(self, name))

    def tu_market_footprint(self, N, M, d, path):
        return 1000

    def tu_market_create(self, *a, **k):
        h = 100 + len(self.created)
        self.created.append(h)
        return h

    def tu_market_destroy(self, h):
        self.destroyed.append(h)

    def tu_market_set_translation(self, h, on):
        pass

    def tu_market_set_relaxation(self, h, omega):
        pass

    def tu_market_update_factors(self, h, *a):
        pass

    def tu_batch_create(self, handles, stream=None):
        from paper_2411_19214_gb300 import TU_ERR_UNSUPPORTED
        raise self.TuError(TU_ERR_UNSUPPORTED, "tu_batch_create")

    def tu_batch_destroy(self, b):
        raise AssertionError("no batch was made")

    def tu_batch_solve(self, *a, **k):
        raise AssertionError("no batch was made")

    def tu_ipfp_solve(self, h, tol, max_iter, warm_start=False):
        from paper_2411_19214_gb300 import TU_ERR_NONFINITE
        self.solved.append(h)
        if h in self.fail:
            raise self.TuError(TU_ERR_NONFINITE, "tu_ipfp_solve")
        return dict(status=0, converged=True, sweeps=3, residual_inf=1e-8, residual_l1=0.0, match_count=7.0)

    def tu_topk_partners(self, h, side, k, row0, nrows, idx, lm):
        idx[:] = np.arange(k, dtype=np.int32)
        lm[:] = 0.0


def test_window_server_solves_a_refused_group_market_by_market(monkeypatch):
    from paper_2411_19214_gb300 import serve
    lib = _FakeLib(serve, monkeypatch)
    reqs = [_req(serve, rid=i) for i in range(3)]
    win = serve.WindowServer(hbm_budget_bytes=1 << 20, tol=1e-6, max_sweeps=50, k=5, max_batch=4)
    res = win.run(reqs, realtime=False)
    assert [r.status for r in res] == ["ok"] * 3 and all(r.sweeps == 3 for r in res)
    assert win.stats["groups"] == 1 and win.stats["solved_alone"] == 3
    assert sorted(lib.solved) == sorted(lib.created) == sorted(lib.destroyed)  # keyless: released after the reply
    assert win.used == 0
    assert all(r.topk_idx.shape == (30, 5) for r in res)


def test_window_server_single_solve_failure_stays_with_its_request(monkeypatch):
    from paper_2411_19214_gb300 import serve
    lib = _FakeLib(serve, monkeypatch, fail={101})
    reqs = [_req(serve, rid=i, key=f"k{i}") for i in range(3)]
    win = serve.WindowServer(hbm_budget_bytes=1 << 20, tol=1e-6, max_sweeps=50, k=5, max_batch=4)
    res = win.run(reqs, realtime=False)
    assert [r.status for r in res] == ["ok", "error", "ok"]
    assert "tu_ipfp_solve" in res[1].error
    # the failed market is released; the others stay resident under their keys
    assert lib.destroyed == [101] and set(win.resident) == {"k0", "k2"}
    assert win.used == 2 * 1000


def test_server_releases_a_market_whose_configuration_fails(monkeypatch):
    """A library error in a call that configures a freshly created market
    (here: switching its graphs off) destroys the market and returns its
    bytes to the budget before the error reaches the request."""
    import torch

    from paper_2411_19214_gb300 import TU_ERR_CUDA, serve
    made, destroyed = [], []
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
    monkeypatch.setattr(serve, "tu_market_create", lambda *a, **k: made.append(7) or 7)
    monkeypatch.setattr(serve, "tu_market_destroy", destroyed.append)

    def fail(h, enable):
        raise serve.TuError(TU_ERR_CUDA, "tu_market_use_graphs")
    monkeypatch.setattr(serve, "tu_market_use_graphs", fail)
    srv = serve.Server(hbm_budget_bytes=1 << 20, tol=1e-6, max_sweeps=50, k=5)
    try:
        srv.used = 1000  # as _admit leaves it for a cold request of 1000 bytes
        req = _req(serve)
        arrays = dict(F=req.F, K=req.K, G=req.G, L=req.L, bias_x=req.bias_x, bias_y=req.bias_y)
        with pytest.raises(serve.TuError):
            srv._activate("cold", 1000, arrays, req, 0.0)
        assert made == [7] and destroyed == [7] and srv.used == 0
    finally:
        srv.pool.shutdown(wait=True)
