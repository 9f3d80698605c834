"""Shared helpers of the GPU parity tests: run the oracle on a synth market."""

import numpy as np

import oracle


def dense_logA(mk):
    f = mk.f64()
    Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"])
    return oracle.log_kernel(Phi, f["sigma"]), f


def oracle_sweeps(mk, sweeps, log_u=None, log_v=None, translate=True):
    """Oracle state after ``sweeps`` sweeps of Eq. iteration from (log_u, log_v),
    each half-sweep preceded by the translation step when ``translate`` (the
    library's default; a market with tu_market_set_translation(m, 0) runs
    Eq. iteration exactly)."""
    logA, f = dense_logA(mk)
    lu = np.zeros(mk.N) if log_u is None else np.asarray(log_u, np.float64)
    lv = np.zeros(mk.M) if log_v is None else np.asarray(log_v, np.float64)
    for _ in range(sweeps):
        if translate:
            lv, lu, _ = oracle.translation_step(lv, lu, f["m"], f["n"])
        lu = oracle.half_sweep_x(logA, lv, f["n"])
        if translate:
            lu, lv, _ = oracle.translation_step(lu, lv, f["n"], f["m"])
        lv = oracle.half_sweep_y(logA, lu, f["m"])
    return lu, lv


def oracle_solve(mk, tol=1e-12, max_sweeps=200000):
    """The oracle's fixed point, reached with its translated iteration (the
    same fixed point as Eq. iteration, pinned in tests/test_oracle.py, in far
    fewer sweeps on balanced markets)."""
    f = mk.f64()
    Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"])
    r = oracle.ipfp_batch(Phi, f["n"], f["m"], f["sigma"], max_sweeps=max_sweeps, tol=tol, translate=True)
    return r, oracle.log_kernel(Phi, f["sigma"]), f
