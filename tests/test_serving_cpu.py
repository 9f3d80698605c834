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
