"""Over-relaxed IPFP on the GPU (an acceleration outside the paper).

Fixed omega: the relaxed sweeps match the oracle's relaxed iterates sweep by
sweep (both paths). Automatic omega: tu_ipfp_solve reaches the oracle's fixed
point of Eq. iteration in fewer sweeps than plain IPFP on a balanced market.
"""

import numpy as np
import pytest

import oracle
from synth import make_market, plain_dense_market

from _parity import dense_logA, oracle_solve

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("path,atol", [("fused", 2e-5), ("dense", 1e-5)])
def test_fixed_omega_iterates_match_oracle(gpu_lib, path, atol):
    tu = gpu_lib
    mk = make_market(600, 450, 32, sigma=0.5, seed=77, bias_x=True, bias_y=True, n_kind="uniform_real",
                     m_kind="uniform_real", dtype="bf16" if path == "fused" else "fp32")
    mkt = tu.from_synth(mk, path=path)
    try:
        mkt.sweep(2)  # plain sweeps first
        lu0, lv0 = (t.double().cpu().numpy() for t in mkt.potentials())
        mkt.set_relaxation(1.5)
        mkt.sweep(4)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        f = mk.f64()
        Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"])
        r = oracle.ipfp_batch(Phi, f["n"], f["m"], f["sigma"], max_sweeps=4, log_u=lu0, log_v=lv0, omega=1.5,
                              translate=True)
        np.testing.assert_allclose(lu, r["log_u"], atol=atol)
        np.testing.assert_allclose(lv, r["log_v"], atol=atol)
    finally:
        mkt.close()


@pytest.mark.parametrize("path", ["fused", "dense"])
def test_automatic_omega_same_fixed_point_fewer_sweeps(gpu_lib, path):
    tu = gpu_lib
    mk = plain_dense_market(N=400, M=400, dtype="bf16" if path == "fused" else "fp32")
    plain = tu.from_synth(mk, path=path)
    fast = tu.from_synth(mk, path=path)
    try:
        # relaxation against Eq. iteration itself: the translation step alone
        # solves this balanced market in a handful of sweeps
        plain.set_translation(False)
        fast.set_translation(False)
        ip = plain.solve(tol=1e-6, max_iter=50000)
        fast.set_relaxation(0.0)
        ifast = fast.solve(tol=1e-6, max_iter=50000)
        assert ip["converged"] and ifast["converged"]
        assert ifast["sweeps"] * 2 < ip["sweeps"], (ifast["sweeps"], ip["sweeps"])
        r, logA, f = oracle_solve(mk, tol=1e-12)
        mu_ref = np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))
        mu = fast.mu_block().double().cpu().numpy()
        print(f"{path}: plain {ip['sweeps']} sweeps, relaxed {ifast['sweeps']}, "
              f"max rel mu err {np.max(np.abs(mu / mu_ref - 1)):.2e}")
        # balanced market: a residual of 1e-6 bounds mu only to ~N * 1e-6
        np.testing.assert_allclose(mu, mu_ref, rtol=1e-3)
        cx = oracle.match_count(f["n"], r["log_u"])
        assert abs(ifast["match_count"] - cx) <= 1e-5 * cx
    finally:
        plain.close()
        fast.close()


def test_invalid_omega_rejected(gpu_lib):
    tu = gpu_lib
    mk = make_market(50, 60, 8, sigma=1.0, seed=1, dtype="bf16")
    mkt = tu.from_synth(mk, path="fused")
    try:
        for bad in (0.5, 2.0, -1.0):
            with pytest.raises(tu.TuError):
                mkt.set_relaxation(bad)
    finally:
        mkt.close()


def test_asynchronous_automatic_omega(gpu_lib):
    """Serving-style loop: blocks of sweeps enqueued with tu_ipfp_sweep, the
    residual read back with tu_market_query, and the automatic controller fed
    between blocks (tu_market_relax_update). Same fixed point, fewer sweeps
    than plain blocks; a relaxation update while a block runs is a no-op."""
    tu = gpu_lib
    mk = plain_dense_market(N=400, M=400, dtype="bf16")

    def run(relax):
        mkt = tu.from_synth(mk, path="fused")
        mkt.set_translation(False)  # relaxation against Eq. iteration itself
        if relax:
            mkt.set_relaxation(0.0)
        done = 0
        while done < 40000:
            tu.tu_ipfp_sweep(mkt.handle, 8)
            done += 8
            while True:
                idle, res, _, sweeps = tu.tu_market_query(mkt.handle)
                if idle:
                    break
                tu.tu_market_relax_update(mkt.handle, 1e-6)  # busy: must not change anything
            assert sweeps == done
            if res <= 1e-6:
                break
            if relax:
                tu.tu_market_relax_update(mkt.handle, 1e-6)
        return mkt, done, res

    plain, n_plain, r_plain = run(False)
    fast, n_fast, r_fast = run(True)
    try:
        assert r_plain <= 1e-6 and r_fast <= 1e-6
        assert n_fast * 2 < n_plain, (n_fast, n_plain)
        r, logA, f = oracle_solve(mk, tol=1e-12)
        mu_ref = np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))
        np.testing.assert_allclose(fast.mu_block().double().cpu().numpy(), mu_ref, rtol=1e-3)
        with pytest.raises(tu.TuError):
            tu.tu_market_relax_update(fast.handle, -1.0)
    finally:
        plain.close()
        fast.close()


@pytest.mark.parametrize("path", ["fused", "dense"])
def test_translation_step_solves_a_balanced_market_in_a_few_sweeps(gpu_lib, path):
    """A balanced 1,000 x 1,000 market with popularity biases on both sides
    (the benchmark's recipe at a size the oracle solves): with the translation
    step (the default) the solve reaches 1e-6 in at most 12 sweeps, where 300
    sweeps of Eq. iteration leave it far from converged; the fixed point is the
    oracle's (mu within the BF16 / FP32 bars, match count within 1e-5)."""
    tu = gpu_lib
    mk = make_market(1000, 1000, 64 if path == "fused" else 32, sigma=0.5, seed=61, bias_x=True, bias_y=True,
                     dtype="bf16" if path == "fused" else "fp32")
    fast = tu.from_synth(mk, path=path)
    plain = tu.from_synth(mk, path=path)
    try:
        info = fast.solve(tol=1e-6, max_iter=1000)
        assert info["converged"] and info["sweeps"] <= 12, info
        plain.set_translation(False)
        ip = plain.solve(tol=1e-6, max_iter=300)
        assert not ip["converged"] and ip["residual_inf"] > 1e-3, ip
        r, logA, f = oracle_solve(mk, tol=1e-12)
        mu_ref = np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))
        mu = fast.mu_block().double().cpu().numpy()
        err = float(np.max(np.abs(mu / mu_ref - 1)))
        cx = oracle.match_count(f["n"], r["log_u"])
        print(f"{path}: translated {info['sweeps']} sweeps (residual {info['residual_inf']:.2e}), plain 300 sweeps "
              f"at {ip['residual_inf']:.2e}; max rel mu err {err:.2e}, match rel err "
              f"{abs(info['match_count'] / cx - 1):.2e}")
        assert err <= (1e-3 if path == "fused" else 1e-5)
        assert abs(info["match_count"] - cx) <= 1e-5 * cx
    finally:
        fast.close()
        plain.close()
