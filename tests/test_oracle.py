"""Pins of the float64 oracle against what the paper and the mathematics fix.

None of these tests uses the CUDA path. Each pin is chosen so that a plausible
mistake in the oracle (a dropped 1/2, beta instead of 2 beta, a transposed
operand, a wrong sign, Jacobi instead of Gauss-Seidel order) fails at least one
of them; ``test_planted_mistakes_are_caught`` checks that for a list of such
mistakes planted into the oracle.
"""

import json
import os

import mpmath as mp
import numpy as np
import pytest

import oracle
from oracle import ipfp as O
from synth import make_market

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _random_market(rng, N, M, d=3, bias=True, cap=True):
    F, K = rng.normal(0, 0.7, (N, d)), rng.normal(0, 0.7, (N, d))
    G, L = rng.normal(0, 0.7, (M, d)), rng.normal(0, 0.7, (M, d))
    bx = rng.lognormal(0, 0.5, N) if bias else None
    by = rng.lognormal(0, 0.5, M) if bias else None
    n = rng.uniform(0.5, 2.0, N) if cap else np.ones(N)
    m = rng.uniform(0.5, 3.0, M) if cap else np.ones(M)
    return F, K, G, L, bx, by, n, m


def _solve(Phi, n, m, beta, tol=1e-13, max_sweeps=200000):
    r = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=max_sweeps, tol=tol)
    assert r["res_inf"] <= tol * 10, r["res_inf"]
    return r


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------

def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _golden()["one_by_one"], ids=lambda c: f"phi{c['phi']}")
def test_closed_form_1x1(case):
    """Eq. stable_condition + Eq. IPFP with one user per side: mu solves
    (a^2-1) mu^2 - a^2 (n+m) mu + a^2 n m = 0, a = exp(phi/(2 beta))."""
    Phi = np.array([[case["phi"]]])
    n, m = np.array([case["n"]]), np.array([case["m"]])
    r = _solve(Phi, n, m, case["beta"], tol=1e-14)
    logA = oracle.log_kernel(Phi, case["beta"])
    mu = float(np.exp(oracle.log_mu(logA, r["log_u"], r["log_v"]))[0, 0])
    exact = float(mp.mpf(case["mu"]))
    assert abs(mu - exact) <= 1e-12 * exact
    # the unmatched masses close the two constraints of Eq. primary optimization
    assert abs(np.exp(2 * r["log_u"][0]) + mu - case["n"]) <= 1e-12 * case["n"]
    assert abs(np.exp(2 * r["log_v"][0]) + mu - case["m"]) <= 1e-12 * case["m"]


def test_closed_form_fixture_matches_formula():
    """The stored 1x1 values are the root of the quadratic (recomputed here)."""
    mp.mp.dps = 40
    for c in _golden()["one_by_one"]:
        a2 = mp.e ** (mp.mpf(str(c["phi"])) / mp.mpf(str(c["beta"])))
        n, m, mu = mp.mpf(str(c["n"])), mp.mpf(str(c["m"])), mp.mpf(c["mu"])
        val = (a2 - 1) * mu ** 2 - a2 * (n + m) * mu + a2 * n * m
        assert abs(val) <= mp.mpf("1e-25") * a2 * n * m


@pytest.mark.parametrize("case", _golden()["symmetric_two_by_two"], ids=lambda c: f"a{c['alpha']}")
def test_closed_form_symmetric_2x2(case):
    """Symmetric 2x2 market, unit capacities: u = v = 1/sqrt(1 + e^{alpha/2b} + e^{gamma/2b})."""
    a, g = case["alpha"], case["gamma"]
    Phi = np.array([[a, g], [g, a]])
    r = _solve(Phi, np.ones(2), np.ones(2), case["beta"], tol=1e-14)
    w = float(mp.mpf(case["w"]))
    np.testing.assert_allclose(np.exp(r["log_u"]), [w, w], rtol=1e-12)
    np.testing.assert_allclose(np.exp(r["log_v"]), [w, w], rtol=1e-12)


# ---------------------------------------------------------------------------
# Independent solvers of the same fixed point
# ---------------------------------------------------------------------------

def _newton_dual(Phi, n, m, beta, iters=100):
    """Maximise the concave dual G(a, b) = sum n a + sum m b - 1/2 sum e^{2a}
    - 1/2 sum e^{2b} - sum_xy A_xy e^{a_x + b_y}, whose gradient is exactly the
    system Eq. IPFP with u = e^a, v = e^b. Newton with backtracking."""
    A = np.exp(Phi / (2 * beta))
    N, M = A.shape

    def value(z):
        a, b = z[:N], z[N:]
        return (n @ a + m @ b - 0.5 * np.sum(np.exp(2 * a)) - 0.5 * np.sum(np.exp(2 * b))
                - np.sum(A * np.exp(a[:, None] + b[None, :])))

    z = np.full(N + M, -1.0)
    for _ in range(iters):
        a, b = z[:N], z[N:]
        mu = A * np.exp(a[:, None] + b[None, :])
        grad = np.concatenate([n - np.exp(2 * a) - mu.sum(1), m - np.exp(2 * b) - mu.sum(0)])
        if np.max(np.abs(grad)) < 1e-15:
            break
        H = np.zeros((N + M, N + M))
        H[:N, :N] = -np.diag(2 * np.exp(2 * a) + mu.sum(1))
        H[N:, N:] = -np.diag(2 * np.exp(2 * b) + mu.sum(0))
        H[:N, N:] = -mu
        H[N:, :N] = -mu.T
        step = np.linalg.solve(H, -grad)
        t, g0 = 1.0, value(z)
        while value(z + t * step) < g0 - 1e-14 and t > 1e-8:
            t *= 0.5
        z = z + t * step
    return z[:N], z[N:]


@pytest.mark.parametrize("shape", [(3, 4), (5, 2), (6, 6)])
def test_newton_on_concave_dual(shape):
    rng = np.random.default_rng(7)
    F, K, G, L, bx, by, n, m = _random_market(rng, *shape)
    beta = 0.8
    Phi = oracle.phi_dense(F, K, G, L, bx, by)
    r = _solve(Phi, n, m, beta)
    a, b = _newton_dual(Phi, n, m, beta)
    np.testing.assert_allclose(r["log_u"], a, atol=1e-11)
    np.testing.assert_allclose(r["log_v"], b, atol=1e-11)


def test_fixed_point_maximises_primal_welfare():
    """Eq. primary optimization: the IPFP equilibrium is the maximiser of
    W = sum mu phi + beta E(mu). W is strictly concave inside the feasible set,
    so a stationary point is the maximum. Check stationarity by central finite
    differences and the maximum against random feasible perturbations. This pins
    the 2 beta of A = exp(Phi / (2 beta)) independently of the iteration."""
    rng = np.random.default_rng(11)
    F, K, G, L, bx, by, n, m = _random_market(rng, 3, 4)
    beta = 0.6
    Phi = oracle.phi_dense(F, K, G, L, bx, by)
    r = _solve(Phi, n, m, beta)
    mu = np.exp(oracle.log_mu(oracle.log_kernel(Phi, beta), r["log_u"], r["log_v"]))
    w0 = oracle.welfare(Phi, mu, n, m, beta)
    h = 1e-6
    for i in range(mu.shape[0]):
        for j in range(mu.shape[1]):
            e = np.zeros_like(mu); e[i, j] = h
            g = (oracle.welfare(Phi, mu + e, n, m, beta) - oracle.welfare(Phi, mu - e, n, m, beta)) / (2 * h)
            assert abs(g) < 1e-6
    for _ in range(200):
        d = rng.normal(size=mu.shape) * 1e-3 * mu
        assert oracle.welfare(Phi, mu + d, n, m, beta) < w0


# ---------------------------------------------------------------------------
# The update and the literal algorithm
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("s", [1e-300, 1e-12, 1e-3, 0.5, 1.0, 7.0, 1e4, 1e8, 1e150, 1e300])
@pytest.mark.parametrize("n", [1e-6, 1.0, 5.0])
def test_scaling_update_against_high_precision(s, n):
    """Eq. iteration: u = sqrt(n + s^2) - s, the printed form evaluated in high precision."""
    # enough digits that the printed difference itself does not cancel
    mp.mp.dps = 60 + int(2 * abs(np.log10(s)) + abs(np.log10(n)))
    S, Nm = mp.mpf(s), mp.mpf(n)
    exact = mp.sqrt(Nm + S * S) - S
    got = oracle.scaling_update(np.log(s), n)  # log u
    assert abs(got - float(mp.log(exact))) <= 1e-13 * max(1.0, abs(got))


def test_printed_update_cancels_where_stable_form_does_not():
    """The printed difference loses every digit once s^2 >> n (reason for the
    stable form); the two agree where it does not cancel."""
    s, n = 1e8, 1.0
    assert np.sqrt(n + s * s) - s == 0.0
    assert np.exp(oracle.scaling_update(np.log(s), n)) == pytest.approx(0.5e-8, rel=1e-12)
    for s in (0.1, 1.0, 3.0):
        assert np.exp(oracle.scaling_update(np.log(s), n)) == pytest.approx(np.sqrt(n + s * s) - s, rel=1e-13)


def test_literal_algorithm_1_matches_log_form():
    """Alg. 1 as printed (linear domain) and the log-domain oracle give the same
    iterates on a well-conditioned market, sweep by sweep."""
    rng = np.random.default_rng(3)
    F, K, G, L, _, _, n, m = _random_market(rng, 7, 5, bias=False)
    beta = 1.0
    P, Q = F @ G.T, K @ L.T
    for iters in (1, 2, 5, 40):
        u, v, mu = oracle.ipfp_batch_literal(P, Q, n, m, beta, iters)
        r = oracle.ipfp_batch(P + Q, n, m, beta, max_sweeps=iters)
        np.testing.assert_allclose(np.log(u), r["log_u"], rtol=0, atol=1e-13)
        np.testing.assert_allclose(np.log(v), r["log_v"], rtol=0, atol=1e-13)
        lm = oracle.log_mu(oracle.log_kernel(P + Q, beta), r["log_u"], r["log_v"])
        np.testing.assert_allclose(np.log(mu), lm, atol=1e-12)


def test_gauss_seidel_order():
    """Eq. iteration: the v step uses the u of the same sweep. One sweep from
    u = v = 1 is checked against values written out by hand for a 1x2 market."""
    Phi = np.array([[0.4, -0.6]])
    beta, n, m = 0.5, np.array([1.0]), np.array([2.0, 1.0])
    A = np.exp(Phi / (2 * beta))[0]
    s = 0.5 * (A[0] + A[1])
    u = np.sqrt(n[0] + s * s) - s
    v = [np.sqrt(m[j] + (0.5 * A[j] * u) ** 2) - 0.5 * A[j] * u for j in range(2)]
    r = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=1)
    assert np.exp(r["log_u"][0]) == pytest.approx(u, rel=1e-14)
    np.testing.assert_allclose(np.exp(r["log_v"]), v, rtol=1e-14)


# ---------------------------------------------------------------------------
# Invariants at the fixed point
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def solved():
    rng = np.random.default_rng(5)
    F, K, G, L, bx, by, n, m = _random_market(rng, 30, 40, d=4)
    beta = 0.7
    Phi = oracle.phi_dense(F, K, G, L, bx, by)
    r = _solve(Phi, n, m, beta)
    return dict(F=F, K=K, G=G, L=L, bx=bx, by=by, n=n, m=m, beta=beta, Phi=Phi, r=r)


def test_marginals_at_fixed_point(solved):
    """Constraints of Eq. primary optimization with mu_x0 = u^2, mu_0y = v^2."""
    s = solved
    logA = oracle.log_kernel(s["Phi"], s["beta"])
    mu = np.exp(oracle.log_mu(logA, s["r"]["log_u"], s["r"]["log_v"]))
    np.testing.assert_allclose(mu.sum(1) + np.exp(2 * s["r"]["log_u"]), s["n"], rtol=1e-12)
    np.testing.assert_allclose(mu.sum(0) + np.exp(2 * s["r"]["log_v"]), s["m"], rtol=1e-12)
    assert oracle.col_residual(logA, s["m"], s["r"]["log_u"], s["r"]["log_v"])[0] < 1e-12


def test_total_mass_identity(solved):
    s = solved
    logA = oracle.log_kernel(s["Phi"], s["beta"])
    mu = np.exp(oracle.log_mu(logA, s["r"]["log_u"], s["r"]["log_v"]))
    cx, cy = oracle.match_count(s["n"], s["r"]["log_u"], s["m"], s["r"]["log_v"])
    assert cx == pytest.approx(mu.sum(), rel=1e-12)
    assert cy == pytest.approx(mu.sum(), rel=1e-12)


def test_permutation_equivariance(solved):
    s = solved
    rng = np.random.default_rng(9)
    px, py = rng.permutation(30), rng.permutation(40)
    Phi = oracle.phi_dense(s["F"][px], s["K"][px], s["G"][py], s["L"][py], s["bx"][px], s["by"][py])
    r = _solve(Phi, s["n"][px], s["m"][py], s["beta"])
    np.testing.assert_allclose(r["log_u"], s["r"]["log_u"][px], atol=1e-11)
    np.testing.assert_allclose(r["log_v"], s["r"]["log_v"][py], atol=1e-11)


def test_side_swap(solved):
    """Exchanging the roles of X and Y (F<->G, K<->L, n<->m) exchanges u and v."""
    s = solved
    Phi_t = oracle.phi_dense(s["G"], s["L"], s["F"], s["K"], s["by"], s["bx"])
    np.testing.assert_allclose(Phi_t, s["Phi"].T, atol=1e-13)
    r = _solve(Phi_t, s["m"], s["n"], s["beta"])
    np.testing.assert_allclose(r["log_u"], s["r"]["log_v"], atol=1e-11)
    np.testing.assert_allclose(r["log_v"], s["r"]["log_u"], atol=1e-11)


def test_mass_scaling(solved):
    """n, m -> c n, c m gives u, v -> sqrt(c) u, sqrt(c) v and mu -> c mu."""
    s = solved
    c = 3.7
    r = _solve(s["Phi"], c * s["n"], c * s["m"], s["beta"])
    np.testing.assert_allclose(r["log_u"], s["r"]["log_u"] + 0.5 * np.log(c), atol=1e-11)
    np.testing.assert_allclose(r["log_v"], s["r"]["log_v"] + 0.5 * np.log(c), atol=1e-11)


def test_constant_shift_is_not_neutral(solved):
    """Adding a constant to phi raises every match gain: the total matched mass
    must grow (the unmatched option is not shifted)."""
    s = solved
    r = _solve(s["Phi"] + 1.0, s["n"], s["m"], s["beta"])
    assert oracle.match_count(s["n"], r["log_u"]) > oracle.match_count(s["n"], s["r"]["log_u"]) + 1e-5
    assert np.min(s["r"]["log_u"] - r["log_u"]) > 0.1  # every unmatched mass shrinks


# ---------------------------------------------------------------------------
# Mini-batch == batch (Sec. 3.3: the mini-batch update needs no approximation)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bx_rows,by_rows", [(1, 1), (3, 7), (7, 40), (31, 2)])
def test_minibatch_iterates_equal_batch(bx_rows, by_rows):
    rng = np.random.default_rng(13)
    F, K, G, L, bx, by, n, m = _random_market(rng, 31, 40, d=4)
    beta = 0.9
    Phi = oracle.phi_dense(F, K, G, L, bx, by)
    for sweeps in (1, 3, 10):
        rb = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=sweeps)
        rm = oracle.ipfp_minibatch(F, K, G, L, n, m, beta, sweeps, bx_rows, by_rows, bx, by)
        np.testing.assert_allclose(rm["log_u"], rb["log_u"], atol=1e-12)
        np.testing.assert_allclose(rm["log_v"], rb["log_v"], atol=1e-12)


# ---------------------------------------------------------------------------
# Stable factors (Psi, Xi)
# ---------------------------------------------------------------------------

def test_stable_factors_corrected_reading(solved):
    """log mu = <psi_x, xi_y>/(2 beta) holds with 2 beta log u, 2 beta log v;
    the printed beta log u, beta log v is off (the garble the reading fixes)."""
    s = solved
    Psi, Xi = oracle.stable_factors(s["F"], s["K"], s["G"], s["L"], s["beta"],
                                    s["r"]["log_u"], s["r"]["log_v"], s["bx"], s["by"])
    assert Psi.shape == (30, 2 * 4 + 2) and Xi.shape == (40, 2 * 4 + 2)
    lm = oracle.log_mu(oracle.log_kernel(s["Phi"], s["beta"]), s["r"]["log_u"], s["r"]["log_v"])
    np.testing.assert_allclose(Psi @ Xi.T / (2 * s["beta"]), lm, atol=1e-12)
    printed_psi = Psi.copy(); printed_xi = Xi.copy()
    printed_psi[:, -2] = s["beta"] * s["r"]["log_u"] + s["bx"]
    printed_xi[:, -1] = s["beta"] * s["r"]["log_v"] + s["by"]
    assert np.max(np.abs(printed_psi @ printed_xi.T / (2 * s["beta"]) - lm)) > 0.1


# ---------------------------------------------------------------------------
# Ranked lists, residual, sampled certification
# ---------------------------------------------------------------------------

def test_topk_against_brute_force():
    rng = np.random.default_rng(17)
    logA = np.round(rng.normal(size=(9, 13)), 1)  # rounded: many exact ties
    lu, lv = np.zeros(9), np.round(rng.normal(size=13), 1) * 0
    for side in (0, 1):
        idx, vals = oracle.topk_partners(logA, lu, lv, 5, side)
        sc = logA if side == 0 else logA.T
        for i in range(sc.shape[0]):
            brute = sorted(range(sc.shape[1]), key=lambda j: (-sc[i, j], j))[:5]
            assert list(idx[i]) == brute
            np.testing.assert_array_equal(vals[i], sc[i, brute])


def test_row_residual_direct():
    rng = np.random.default_rng(19)
    F, K, G, L, bx, by, n, m = _random_market(rng, 6, 8)
    beta = 1.1
    Phi = oracle.phi_dense(F, K, G, L, bx, by)
    lu, lv = rng.normal(size=6) - 1, rng.normal(size=8) - 1
    A = np.exp(Phi / (2 * beta))
    u, v = np.exp(lu), np.exp(lv)
    r_direct = u * u + u * (A @ v) - n
    r_inf, r_l1, r = oracle.row_residual(oracle.log_kernel(Phi, beta), n, lu, lv)
    np.testing.assert_allclose(r, r_direct, rtol=1e-12)
    assert r_inf == pytest.approx(np.max(np.abs(r_direct) / n), rel=1e-12)
    assert r_l1 == pytest.approx(np.sum(np.abs(r_direct)) / np.sum(n), rel=1e-12)


def test_col_residual_direct():
    """The column equations of Eq. IPFP written out in the linear domain,
    m_y = v_y^2 + v_y sum_x A_xy u_x, at arbitrary potentials; and zero (to
    rounding) right after a Y half-sweep, which solves exactly those
    equations for v."""
    rng = np.random.default_rng(29)
    F, K, G, L, bx, by, n, m = _random_market(rng, 7, 5)
    beta = 0.8
    Phi = oracle.phi_dense(F, K, G, L, bx, by)
    lu, lv = rng.normal(size=7) - 1, rng.normal(size=5) - 1
    A = np.exp(Phi / (2 * beta))
    u, v = np.exp(lu), np.exp(lv)
    r_direct = v * v + v * (A.T @ u) - m
    logA = oracle.log_kernel(Phi, beta)
    r_inf, r_l1, r = oracle.col_residual(logA, m, lu, lv)
    np.testing.assert_allclose(r, r_direct, rtol=1e-12)
    assert r_inf == pytest.approx(np.max(np.abs(r_direct) / m), rel=1e-12)
    assert r_l1 == pytest.approx(np.sum(np.abs(r_direct)) / np.sum(m), rel=1e-12)
    lv_new = oracle.half_sweep_y(logA, lu, m)
    assert oracle.col_residual(logA, m, lu, lv_new)[0] < 1e-13


def test_sampled_row_update_equals_dense_half_sweep():
    mk = make_market(50, 333, 8, sigma=0.5, seed=23, bias_x=True, bias_y=True, dtype="bf16")
    f = mk.f64()
    Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"])
    logA = oracle.log_kernel(Phi, f["sigma"])
    lv = np.random.default_rng(1).normal(size=333)
    full = oracle.half_sweep_x(logA, lv, f["n"])
    rows = np.array([0, 7, 19, 49])
    _, lu = oracle.sampled_row_update(f["F"], f["K"], f["G"], f["L"], f["sigma"], f["n"], lv, rows,
                                      f["bias_x"], f["bias_y"], col_chunk=50)
    np.testing.assert_allclose(lu, full[rows], atol=1e-13)
    # the Y side through the same function with the sides exchanged
    lu_all = full
    fully = oracle.half_sweep_y(logA, lu_all, f["m"])
    cols = np.array([3, 100, 332])
    _, lvs = oracle.sampled_row_update(f["G"], f["L"], f["F"], f["K"], f["sigma"], f["m"], lu_all, cols,
                                       f["bias_y"], f["bias_x"], col_chunk=17)
    np.testing.assert_allclose(lvs, fully[cols], atol=1e-13)


# ---------------------------------------------------------------------------
# The pins catch plausible mistakes
# ---------------------------------------------------------------------------

def _pins_pass():
    """Run a compact set of the pins above; True if all hold."""
    try:
        g = _golden()
        for c in g["one_by_one"][:3]:
            test_closed_form_1x1(c)
        for c in g["symmetric_two_by_two"]:
            test_closed_form_symmetric_2x2(c)
        test_fixed_point_maximises_primal_welfare()
        test_gauss_seidel_order()
        test_literal_algorithm_1_matches_log_form()
        test_row_residual_direct()
        test_newton_on_concave_dual((6, 6))
    except (AssertionError, ValueError, FloatingPointError):
        return False
    return True


MISTAKES = {
    "drop the 1/2 in s = A v / 2": ("LOG_HALF", 0.0),
    "beta instead of 2 beta": ("log_kernel", lambda Phi, beta: np.asarray(Phi, float) / float(beta)),
    "wrong sign in the update": ("scaling_update",
                                 lambda log_s, mass: 0.5 * np.log(mass) + O.asinh_exp(log_s - 0.5 * np.log(mass))),
    "transposed kernel in the u step": ("half_sweep_x",
                                        lambda logA, lv, n: O.scaling_update(
                                            O.LOG_HALF + O._logsumexp(logA.T + lv[None, :], axis=1), n)),
    "Jacobi order (v from the old u)": None,
    "residual without the u^2 term": ("row_residual", None),
}


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_pass()
    for name, patch in MISTAKES.items():
        with monkeypatch.context() as mpatch:
            if name.startswith("Jacobi"):
                orig_batch = O.ipfp_batch

                def jacobi(Phi, n, m, beta, max_sweeps, tol=None, log_u=None, log_v=None):
                    logA = O.log_kernel(Phi, beta)
                    lu = np.zeros(logA.shape[0]) if log_u is None else log_u
                    lv = np.zeros(logA.shape[1]) if log_v is None else log_v
                    for _ in range(int(max_sweeps)):
                        if tol is not None and O.row_residual(logA, n, lu, lv)[0] <= tol:
                            break
                        lu, lv = O.half_sweep_x(logA, lv, n), O.half_sweep_y(logA, lu, m)
                    r = orig_batch(Phi, n, m, beta, 0, None, lu, lv)
                    return r
                mpatch.setattr(O, "ipfp_batch", jacobi)
                mpatch.setattr(oracle, "ipfp_batch", jacobi)
            elif name.startswith("residual"):
                def bad_res(logA, n, log_u, log_v):
                    lse = O._logsumexp(logA + log_v[None, :], axis=1)
                    r = np.exp(log_u + lse) - n
                    return float(np.max(np.abs(r) / n)), float(np.sum(np.abs(r)) / np.sum(n)), r
                mpatch.setattr(O, "row_residual", bad_res)
                mpatch.setattr(oracle, "row_residual", bad_res)
            else:
                attr, val = patch
                mpatch.setattr(O, attr, val)
                if hasattr(oracle, attr):
                    mpatch.setattr(oracle, attr, val)
            assert not _pins_pass(), f"planted mistake not caught: {name}"
    assert _pins_pass()


# ---------------------------------------------------------------------------
# Over-relaxed iteration (an extension): same fixed point, fewer sweeps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("omega", [1.3, 1.6, 1.8])
def test_relaxed_iteration_reaches_the_dual_fixed_point(omega):
    rng = np.random.default_rng(29)
    F, K, G, L, bx, by, n, m = _random_market(rng, 6, 6)
    beta = 0.8
    Phi = oracle.phi_dense(F, K, G, L, bx, by)
    r = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=100000, tol=1e-13, omega=omega)
    assert r["res_inf"] <= 1e-12
    a, b = _newton_dual(Phi, n, m, beta)
    np.testing.assert_allclose(r["log_u"], a, atol=1e-11)
    np.testing.assert_allclose(r["log_v"], b, atol=1e-11)


def test_relaxed_iteration_one_sweep_by_hand():
    """One relaxed sweep = plain update u', then log u + omega (log u' - log u),
    and the v update uses the relaxed u."""
    Phi = np.array([[0.4, -0.6], [1.0, 0.2]])
    beta, n, m, om = 0.5, np.array([1.0, 2.0]), np.array([2.0, 1.0]), 1.7
    lu0, lv0 = np.array([-0.3, 0.1]), np.array([0.2, -0.5])
    logA = oracle.log_kernel(Phi, beta)
    A = np.exp(logA)
    s = 0.5 * A @ np.exp(lv0)
    lu_plain = np.log(np.sqrt(n + s * s) - s)
    lu = lu0 + om * (lu_plain - lu0)
    s = 0.5 * A.T @ np.exp(lu)
    lv_plain = np.log(np.sqrt(m + s * s) - s)
    lv = lv0 + om * (lv_plain - lv0)
    r = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=1, log_u=lu0, log_v=lv0, omega=om)
    np.testing.assert_allclose(r["log_u"], lu, atol=1e-14)
    np.testing.assert_allclose(r["log_v"], lv, atol=1e-14)


def test_relaxation_cuts_sweeps_on_a_balanced_market():
    mk = make_market(100, 100, 16, sigma=1.0, seed=100, dtype="fp32")
    f = mk.f64()
    Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"])
    plain = oracle.ipfp_batch(Phi, f["n"], f["m"], 1.0, max_sweeps=20000, tol=1e-8)
    fast = oracle.ipfp_batch(Phi, f["n"], f["m"], 1.0, max_sweeps=20000, tol=1e-8, omega=1.6)
    assert fast["sweeps"] * 2 < plain["sweeps"]
    np.testing.assert_allclose(fast["log_u"], plain["log_u"], atol=1e-6)


# ---------------------------------------------------------------------------
# Translation step (an extension): exact line search of the dual
# ---------------------------------------------------------------------------

def _line_argmax(f, lo=-40.0, hi=40.0):
    """Brute-force maximiser of a concave function of one variable: a grid,
    then golden-section search on the bracket around the best grid point."""
    ts = np.linspace(lo, hi, 4001)
    vals = [f(t) for t in ts]
    i = int(np.argmax(vals))
    a, b = ts[max(i - 1, 0)], ts[min(i + 1, len(ts) - 1)]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(200):
        if f(c) > f(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    return 0.5 * (a + b)


@pytest.mark.parametrize("seed,shape,cap", [(41, (5, 7), True), (42, (6, 3), True), (43, (4, 4), False)])
def test_translation_step_maximises_the_dual_on_its_line(seed, shape, cap):
    """The closed-form tau is the maximiser of the full dual (pair sum
    included) along (log u + tau, log v - tau), found by brute force, and
    the dual rises."""
    rng = np.random.default_rng(seed)
    F, K, G, L, bx, by, n, m = _random_market(rng, *shape, cap=cap)
    beta = 0.7
    logA = oracle.log_kernel(oracle.phi_dense(F, K, G, L, bx, by), beta)
    lu = rng.normal(-1.0, 0.8, shape[0])
    lv = rng.normal(-2.5, 0.8, shape[1])
    lu2, lv2, tau = oracle.translation_step(lu, lv, n, m)
    t_bf = _line_argmax(lambda t: oracle.dual_value(logA, n, m, lu + t, lv - t))
    assert abs(tau - t_bf) < 1e-7, (tau, t_bf)
    np.testing.assert_allclose(lu2, lu + tau, atol=0)
    np.testing.assert_allclose(lv2, lv - tau, atol=0)
    assert oracle.dual_value(logA, n, m, lu2, lv2) >= oracle.dual_value(logA, n, m, lu, lv)
    # with the sides exchanged the step is the same move
    lv3, lu3, tau_y = oracle.translation_step(lv, lu, m, n)
    assert abs(tau_y + tau) < 1e-12


def test_translation_step_equalises_the_match_counts():
    """At the step's optimum the derivative along the line, summed Eq. IPFP
    rows minus summed columns, vanishes: sum n - sum u^2 = sum m - sum v^2."""
    rng = np.random.default_rng(44)
    for N, M in [(30, 20), (20, 30), (25, 25)]:
        n = rng.uniform(0.2, 3.0, N)
        m = rng.uniform(0.2, 3.0, M)
        lu = rng.normal(0.5, 2.0, N)
        lv = rng.normal(-3.0, 2.0, M)
        lu2, lv2, _ = oracle.translation_step(lu, lv, n, m)
        cx, cy = oracle.match_count(n, lu2, m, lv2)
        assert abs(cx - cy) <= 1e-12 * (np.sum(n) + np.sum(m)), (cx, cy)


@pytest.mark.parametrize("center_p,center_o,dm", [(0.0, 0.0, 0.0), (150.0, -200.0, 3.0), (-300.0, 250.0, -2.0),
                                                  (-20.0, -25.0, 2.0 ** -30), (5.0, 4.0, -7.5)])
def test_translation_step_against_high_precision(center_p, center_o, dm):
    """tau against the positive root of P z^2 - Dm z - O = 0 solved with
    60 significant digits, on potentials whose squares over- or underflow
    float64 and for both signs of the mass difference."""
    rng = np.random.default_rng(45)
    lp = center_p + rng.normal(0.0, 1.0, 6)
    lo = center_o + rng.normal(0.0, 1.0, 6)
    # dyadic capacities: both sums, and so the mass difference, are exact in float64
    mass_o = rng.integers(8, 17, 5) / 8.0
    mass_p = np.concatenate([rng.integers(1, 5, 5) / 8.0, [0.0]])
    mass_p[5] = np.sum(mass_o) + dm - np.sum(mass_p[:5]) + 8.0
    mass_o = np.concatenate([mass_o, [8.0]])
    dm_exact = mp.fsum([mp.mpf(float(x)) for x in mass_p]) - mp.fsum([mp.mpf(float(x)) for x in mass_o])
    _, _, tau = oracle.translation_step(lp, lo, mass_p, mass_o)
    mp.mp.dps = 60
    P = mp.fsum([mp.e ** (2 * mp.mpf(float(x))) for x in lp])
    O_ = mp.fsum([mp.e ** (2 * mp.mpf(float(x))) for x in lo])
    z = (dm_exact + mp.sqrt(dm_exact ** 2 + 4 * P * O_)) / (2 * P)
    tau_exact = mp.log(z) / 2
    assert abs(tau - float(tau_exact)) <= 1e-12 * max(1.0, abs(float(tau_exact))), (tau, tau_exact)


@pytest.mark.parametrize("shape", [(3, 4), (6, 6), (7, 2)])
def test_translated_iteration_reaches_the_dual_fixed_point(shape):
    rng = np.random.default_rng(46)
    F, K, G, L, bx, by, n, m = _random_market(rng, *shape)
    beta = 0.8
    Phi = oracle.phi_dense(F, K, G, L, bx, by)
    r = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=100000, tol=1e-13, translate=True)
    assert r["res_inf"] <= 1e-12
    a, b = _newton_dual(Phi, n, m, beta)
    np.testing.assert_allclose(r["log_u"], a, atol=1e-11)
    np.testing.assert_allclose(r["log_v"], b, atol=1e-11)


def test_translated_sweep_by_hand():
    """One translated sweep of a 2x2 market written out in the linear domain:
    v e^{tau}, u e^{-tau} with z = e^{2 tau} the positive root of
    (sum v^2) z^2 - (sum m - sum n) z - sum u^2 = 0; the printed u update;
    u e^{tau'}, v e^{-tau'} with the roles exchanged; the printed v update."""
    Phi = np.array([[0.4, -0.6], [1.0, 0.2]])
    beta, n, m = 0.5, np.array([1.0, 2.0]), np.array([2.5, 1.0])
    u, v = np.exp(np.array([-0.3, 0.1])), np.exp(np.array([0.2, -0.5]))
    A = np.exp(Phi / (2 * beta))

    def root(p2, o2, dmass):
        return (dmass + np.sqrt(dmass * dmass + 4 * p2 * o2)) / (2 * p2)

    z = root(np.sum(v * v), np.sum(u * u), np.sum(m) - np.sum(n))
    v, u = v * np.sqrt(z), u / np.sqrt(z)
    s = 0.5 * A @ v
    u = np.sqrt(n + s * s) - s
    z = root(np.sum(u * u), np.sum(v * v), np.sum(n) - np.sum(m))
    u, v = u * np.sqrt(z), v / np.sqrt(z)
    s = 0.5 * A.T @ u
    v = np.sqrt(m + s * s) - s
    r = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=1, log_u=np.array([-0.3, 0.1]),
                          log_v=np.array([0.2, -0.5]), translate=True)
    np.testing.assert_allclose(np.exp(r["log_u"]), u, rtol=1e-13)
    np.testing.assert_allclose(np.exp(r["log_v"]), v, rtol=1e-13)


def test_translated_iteration_ascends_the_dual():
    """Every half-sweep and every translation step raises the dual."""
    mk = make_market(40, 40, 8, sigma=0.5, seed=47, bias_x=True, bias_y=True, dtype="fp32")
    f = mk.f64()
    logA = oracle.log_kernel(oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"]), 0.5)
    n, m = f["n"], f["m"]
    lu, lv = np.zeros(40), np.zeros(40)
    prev = oracle.dual_value(logA, n, m, lu, lv)
    for _ in range(6):
        for step in ("ty", "x", "tx", "y"):
            if step == "ty":
                lv, lu, _ = oracle.translation_step(lv, lu, m, n)
            elif step == "x":
                lu = oracle.half_sweep_x(logA, lv, n)
            elif step == "tx":
                lu, lv, _ = oracle.translation_step(lu, lv, n, m)
            else:
                lv = oracle.half_sweep_y(logA, lu, m)
            cur = oracle.dual_value(logA, n, m, lu, lv)
            assert cur >= prev - 1e-9 * abs(prev), (step, cur, prev)
            prev = cur


def test_translation_cuts_sweeps_on_a_balanced_market():
    """The slow mode of a balanced market is the translation itself: with the
    step, a 200 x 200 market with popularity biases reaches 1e-8 in a handful
    of sweeps instead of thousands, at the same fixed point."""
    mk = make_market(200, 200, 16, sigma=0.5, seed=48, bias_x=True, bias_y=True, dtype="fp32")
    f = mk.f64()
    Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"])
    fast = oracle.ipfp_batch(Phi, f["n"], f["m"], 0.5, max_sweeps=200, tol=1e-8, translate=True)
    assert fast["res_inf"] <= 1e-8 and fast["sweeps"] <= 12, fast["sweeps"]
    plain = oracle.ipfp_batch(Phi, f["n"], f["m"], 0.5, max_sweeps=200, tol=1e-8)
    assert plain["res_inf"] > 1e-3  # still far from it after 200 plain sweeps
    a, b = _newton_dual(Phi, f["n"], f["m"], 0.5, iters=200)
    np.testing.assert_allclose(fast["log_u"], a, atol=1e-7)
    np.testing.assert_allclose(fast["log_v"], b, atol=1e-7)


_TRANSLATION_STEP = O.translation_step


def _bad_same_sign(lp, lo, mass_p, mass_o):
    _, _, tau = _TRANSLATION_STEP(lp, lo, mass_p, mass_o)
    return np.asarray(lp) + tau, np.asarray(lo) + tau, tau


def _bad_no_half(lp, lo, mass_p, mass_o):
    _, _, tau = _TRANSLATION_STEP(lp, lo, mass_p, mass_o)
    return np.asarray(lp) + 2 * tau, np.asarray(lo) - 2 * tau, 2 * tau


def _bad_masses_exchanged(lp, lo, mass_p, mass_o):
    return _TRANSLATION_STEP(lp, lo, mass_o, mass_p)


def _bad_other_root(lp, lo, mass_p, mass_o):
    P = np.sum(np.exp(2 * np.asarray(lp)))
    Oo = np.sum(np.exp(2 * np.asarray(lo)))
    dm = float(np.sum(mass_p) - np.sum(mass_o))
    tau = 0.5 * np.log(abs((dm - np.sqrt(dm * dm + 4 * P * Oo)) / (2 * P)))
    return np.asarray(lp) + tau, np.asarray(lo) - tau, tau


TRANSLATION_MISTAKES = {
    "tau applied with the same sign to both sides": _bad_same_sign,
    "tau without the 1/2 (log z)": _bad_no_half,
    "masses of the two sides exchanged": _bad_masses_exchanged,
    "the other root of the quadratic (its magnitude)": _bad_other_root,
}


def _translation_pins_pass():
    try:
        for args in [(41, (5, 7), True), (43, (4, 4), False)]:
            test_translation_step_maximises_the_dual_on_its_line(*args)
        test_translation_step_equalises_the_match_counts()
        test_translated_sweep_by_hand()
        test_translated_iteration_reaches_the_dual_fixed_point((3, 4))
    except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError):
        return False
    return True


def test_planted_translation_mistakes_are_caught(monkeypatch):
    assert _translation_pins_pass()
    for name, bad in TRANSLATION_MISTAKES.items():
        with monkeypatch.context() as mpatch:
            mpatch.setattr(O, "translation_step", bad)
            mpatch.setattr(oracle, "translation_step", bad)
            assert not _translation_pins_pass(), f"planted mistake not caught: {name}"
    assert _translation_pins_pass()


# ---------------------------------------------------------------------------
# Jacobi order (an extension): both half-sweeps from the entering state
# ---------------------------------------------------------------------------

def test_jacobi_one_sweep_by_hand():
    """1x2 market from u = v = 1: u' from the old v, v' from the old u = 1
    (Gauss-Seidel would use the new u), written out by hand."""
    Phi = np.array([[0.4, -0.6]])
    beta, n, m = 0.5, np.array([1.0]), np.array([2.0, 1.0])
    A = np.exp(Phi / (2 * beta))[0]
    s = 0.5 * (A[0] + A[1])
    u = np.sqrt(n[0] + s * s) - s
    v = [np.sqrt(m[j] + (0.5 * A[j]) ** 2) - 0.5 * A[j] for j in range(2)]
    r = oracle.ipfp_jacobi(Phi, n, m, beta, max_sweeps=1)
    assert np.exp(r["log_u"][0]) == pytest.approx(u, rel=1e-14)
    np.testing.assert_allclose(np.exp(r["log_v"]), v, rtol=1e-14)
    gs = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=1)
    assert abs(gs["log_v"][0] - r["log_v"][0]) > 1e-3  # not the Gauss-Seidel order


@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_jacobi_is_two_interleaved_gauss_seidel_runs(k):
    """Jacobi states (U_t, V_t), U_{t+1} = f(V_t), V_{t+1} = g(U_t), hold two
    independent Gauss-Seidel sequences: started from v_0, k Gauss-Seidel
    sweeps give (U_{2k-1}, V_{2k}); started from v = g(u_0) = V_1, they give
    (U_{2k}, V_{2k+1}). Bit for bit: the same half-sweeps in the same order."""
    rng = np.random.default_rng(40 + k)
    F, K, G, L, bx, by, n, m = _random_market(rng, 9, 7)
    Phi = oracle.phi_dense(F, K, G, L, bx, by)
    beta = 0.8
    u0, v0 = rng.normal(0, 0.5, 9), rng.normal(0, 0.5, 7)
    jac = oracle.ipfp_jacobi(Phi, n, m, beta, max_sweeps=2 * k + 1, log_u=u0, log_v=v0)
    S = [(u0, v0)] + jac["states"]
    a = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=k, log_u=u0, log_v=v0)
    np.testing.assert_array_equal(a["log_u"], S[2 * k - 1][0])
    np.testing.assert_array_equal(a["log_v"], S[2 * k][1])
    b = oracle.ipfp_batch(Phi, n, m, beta, max_sweeps=k, log_u=u0, log_v=S[1][1])
    np.testing.assert_array_equal(b["log_u"], S[2 * k][0])
    np.testing.assert_array_equal(b["log_v"], S[2 * k + 1][1])


def test_jacobi_same_fixed_point_twice_the_sweeps():
    """Consequence of the interleaving: the Jacobi order reaches the fixed
    point of Eq. IPFP, and needs at least twice the sweeps of Gauss-Seidel to
    the same residual (measured 2.0-2.5: its state pairs the u of one chain
    with the v of the other), so halving the pair work of a sweep would at best
    break even."""
    ratios = []
    for seed in (1, 2, 3):
        rng = np.random.default_rng(seed)
        F, K, G, L, bx, by, n, m = _random_market(rng, 40, 30, cap=seed != 3)
        Phi = oracle.phi_dense(F, K, G, L, bx, by)
        gs = oracle.ipfp_batch(Phi, n, m, 1.0, max_sweeps=100000, tol=1e-10)
        jac = oracle.ipfp_jacobi(Phi, n, m, 1.0, max_sweeps=200000, tol=1e-10)
        assert jac["res_inf"] <= 1e-10
        np.testing.assert_allclose(jac["log_u"], gs["log_u"], atol=1e-8)
        np.testing.assert_allclose(jac["log_v"], gs["log_v"], atol=1e-8)
        ratios.append(jac["sweeps"] / gs["sweeps"])
    assert all(r >= 1.9 for r in ratios), ratios
