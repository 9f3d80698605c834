"""Float64 IPFP for the Choo-Siow transferable-utility matching model.

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy, float64,
no blocking, fusion or reordering beyond what the cited passage states.

Notation follows the paper's main text (Sec. 3): side X (candidates, index x,
capacities n_x) and side Y (employers, index y, capacities m_y); beta > 0 is the
entropy scale; Phi is the joint surplus phi_xy = p_xy + q_yx; A = exp(Phi/(2 beta));
u_x = sqrt(mu_x0), v_y = sqrt(mu_0y). Alg. 1 and Alg. 2 name the capacity
vectors the other way round (m for X, n for Y); this module keeps the main-text
names everywhere.

Scaling vectors are carried as logarithms (log u, log v) so that markets whose
surplus spans hundreds of nats stay representable; every update is the
algebraically identical form of the printed one (reading stated per function).
"""

from __future__ import annotations

import numpy as np

LOG_HALF = float(np.log(0.5))


# ---------------------------------------------------------------------------
# Surplus and kernel
# ---------------------------------------------------------------------------

def phi_dense(F, K, G, L, bias_x=None, bias_y=None):
    """Joint surplus Phi (N x M).

    Sec. 3.3, Eq. for p and q: p_xy = <f_x, g_y> and q_yx = <k_x, l_y>; Sec. 3.1:
    phi_xy = p_xy + q_yx. So Phi = F G^T + K L^T (the numerator of A_j in
    Eq. iteration_minibatch, taken over all rows).

    Reading (popularity biases, not in the paper): optional per-user additive
    terms, phi_xy += bias_x[x] + bias_y[y], with unit coefficient.
    """
    F = np.asarray(F, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    P = F @ G.T
    Q = K @ L.T
    Phi = P + Q
    if bias_x is not None:
        Phi = Phi + np.asarray(bias_x, dtype=np.float64)[:, None]
    if bias_y is not None:
        Phi = Phi + np.asarray(bias_y, dtype=np.float64)[None, :]
    return Phi


def log_kernel(Phi, beta):
    """log A with A = exp(Phi / (2 beta)) (Eq. iteration_matrix, definition of A;
    Alg. 1, construction of A)."""
    return np.asarray(Phi, dtype=np.float64) / (2.0 * float(beta))


def _logsumexp(a, axis):
    """log(sum(exp(a))) along ``axis`` with the maximum factored out."""
    mx = np.max(a, axis=axis, keepdims=True)
    out = np.log(np.sum(np.exp(a - mx), axis=axis, keepdims=True)) + mx
    return np.squeeze(out, axis=axis)


# ---------------------------------------------------------------------------
# The closed-form per-user update
# ---------------------------------------------------------------------------

def asinh_exp(z):
    """asinh(exp(z)) for any real z, without overflow.

    For z > 0: asinh(e^z) = log(e^z + sqrt(e^{2z} + 1)) = z + log(1 + sqrt(1 + e^{-2z})).
    For z <= 0: e^z <= 1 and asinh is evaluated directly.
    """
    z = np.asarray(z, dtype=np.float64)
    pos = z + np.log1p(np.sqrt(1.0 + np.exp(-2.0 * np.abs(z))))
    neg = np.arcsinh(np.exp(np.minimum(z, 0.0)))
    return np.where(z > 0, pos, neg)


def scaling_update(log_s, mass):
    """Eq. iteration: u = sqrt(n + s^2) - s, returned as log u.

    Reading: the printed difference cancels catastrophically when s^2 >> n, so
    the algebraically identical form is used:
        sqrt(n + s^2) - s = n / (s + sqrt(n + s^2)) = sqrt(n) / (t + sqrt(1 + t^2))
                          = sqrt(n) * exp(-asinh(t)),   t = s / sqrt(n),
    i.e. log u = (1/2) log n - asinh(exp(log s - (1/2) log n)).
    """
    half_log_mass = 0.5 * np.log(np.asarray(mass, dtype=np.float64))
    return half_log_mass - asinh_exp(np.asarray(log_s, dtype=np.float64) - half_log_mass)


def half_sweep_x(logA, log_v, n):
    """First line of Eq. iteration / Eq. iteration_matrix (Alg. 1, the u step):
    s = A v / 2, then u = sqrt(n + s^2) - s, in logs:
    log s_x = log(1/2) + log sum_y exp(log A_xy + log v_y)."""
    log_s = LOG_HALF + _logsumexp(logA + log_v[None, :], axis=1)
    return scaling_update(log_s, n)


def half_sweep_y(logA, log_u, m):
    """Second line of Eq. iteration / Eq. iteration_matrix (Alg. 1, the v step),
    with the u just computed (Gauss-Seidel order): s = A^T u / 2, then
    v = sqrt(m + s^2) - s."""
    log_s = LOG_HALF + _logsumexp(logA + log_u[:, None], axis=0)
    return scaling_update(log_s, m)


# ---------------------------------------------------------------------------
# Residual of the fixed-point equations
# ---------------------------------------------------------------------------

def row_residual(logA, n, log_u, log_v):
    """Residual of the row equations of Eq. IPFP:
        r_x = u_x^2 + u_x * sum_y A_xy v_y - n_x      (u^2 = mu_x0, v^2 = mu_0y).

    Reading (the paper runs a fixed number of iterations and states no
    stopping rule): convergence is measured by
        res_inf = max_x |r_x| / n_x     and     res_l1 = sum_x |r_x| / sum_x n_x.
    After a full sweep the column equations hold up to rounding, so only rows
    are measured. Returns (res_inf, res_l1, r).
    """
    n = np.asarray(n, dtype=np.float64)
    lse = _logsumexp(logA + log_v[None, :], axis=1)
    r = np.exp(2.0 * log_u) + np.exp(log_u + lse) - n
    return float(np.max(np.abs(r) / n)), float(np.sum(np.abs(r)) / np.sum(n)), r


def col_residual(logA, m, log_u, log_v):
    """Residual of the column equations of Eq. IPFP (second line), same measure."""
    m = np.asarray(m, dtype=np.float64)
    lse = _logsumexp(logA + log_u[:, None], axis=0)
    r = np.exp(2.0 * log_v) + np.exp(log_v + lse) - m
    return float(np.max(np.abs(r) / m)), float(np.sum(np.abs(r)) / np.sum(m)), r


# ---------------------------------------------------------------------------
# Translation step (an extension: exact line search of the dual)
# ---------------------------------------------------------------------------

def dual_value(logA, n, m, log_u, log_v):
    """The concave function whose stationarity conditions are Eq. IPFP:
        D(a, b) = sum_x n_x a_x + sum_y m_y b_y - 1/2 sum_x e^{2 a_x} - 1/2 sum_y e^{2 b_y}
                  - sum_xy A_xy e^{a_x + b_y},     a = log u, b = log v.
    d D / d a_x = n_x - u_x^2 - u_x sum_y A_xy v_y is the first line of Eq. IPFP
    (and d D / d b_y the second), so IPFP, which solves the row equations and
    then the column equations exactly, is block coordinate ascent on D
    (Sec. 3.1 describes IPFP as a coordinate method on the dual of
    Eq. primary optimization). Evaluated with the maximum factored out of
    the pair sum."""
    lu = np.asarray(log_u, np.float64)
    lv = np.asarray(log_v, np.float64)
    pair = logA + lu[:, None] + lv[None, :]
    mx = np.max(pair)
    return float(np.dot(n, lu) + np.dot(m, lv) - 0.5 * np.sum(np.exp(2.0 * lu)) - 0.5 * np.sum(np.exp(2.0 * lv))
                 - np.exp(mx) * np.sum(np.exp(pair - mx)))


def translation_step(log_p, log_o, mass_p, mass_o):
    """Exact maximisation of ``dual_value`` along (log p + tau, log o - tau).

    Not in the paper (Sec. 5 names acceleration techniques from optimal
    transport as future work). Moving one side's log potentials up by tau and
    the other side's down by tau leaves every pair term A_xy u_x v_y unchanged,
    so along that line the dual is
        D(tau) = const + tau (sum mass_p - sum mass_o) - 1/2 e^{2 tau} P - 1/2 e^{-2 tau} O,
    P = sum e^{2 log p}, O = sum e^{2 log o}. D is strictly concave in tau and
    D'(tau) = 0 is, with z = e^{2 tau} > 0, the quadratic
        P z^2 - Dm z - O = 0,   Dm = sum mass_p - sum mass_o,
    whose positive root is z = (Dm + R) / (2 P) = 2 O / (R - Dm),
    R = sqrt(Dm^2 + 4 P O). The first form is used for Dm >= 0 and the second
    for Dm < 0, so no subtraction cancels; P and O are carried as logarithms
    (log-sum-exp), so potentials of any size are handled.
    At the returned point sum mass_p - P' = sum mass_o - O': the two forms of
    the match count (Eq. IPFP summed over each side) agree.

    Returns (log_p + tau, log_o - tau, tau).
    """
    lp = np.asarray(log_p, np.float64)
    lo = np.asarray(log_o, np.float64)
    log_P = _logsumexp(2.0 * lp, axis=0)
    log_O = _logsumexp(2.0 * lo, axis=0)
    dm = float(np.sum(mass_p) - np.sum(mass_o))
    log_4po = np.log(4.0) + log_P + log_O
    log_R = 0.5 * (np.logaddexp(2.0 * np.log(abs(dm)), log_4po) if dm != 0.0 else log_4po)
    if dm >= 0.0:
        log_num = np.logaddexp(np.log(dm), log_R) if dm > 0.0 else log_R
        log_z = log_num - np.log(2.0) - log_P
    else:
        log_z = np.log(2.0) + log_O - np.logaddexp(log_R, np.log(-dm))
    tau = 0.5 * float(log_z)
    return lp + tau, lo - tau, tau


# ---------------------------------------------------------------------------
# Batch IPFP (Alg. 1)
# ---------------------------------------------------------------------------

def ipfp_batch(Phi, n, m, beta, max_sweeps, tol=None, log_u=None, log_v=None, omega=1.0, translate=False):
    """Batch IPFP, Alg. 1 / Eq. iteration_matrix, in logs.

    Starts from u = v = 1 (Alg. 1 initialisation) unless a warm start
    (log_u, log_v) is given. Each sweep updates u from v, then v from the new u.
    If ``tol`` is given, the row residual of the current state is evaluated
    before every sweep and the loop stops as soon as res_inf <= tol.

    omega != 1 (an extension, not in the paper) over-relaxes each update in
    the log domain, log u <- log u + omega * (update - log u), and likewise for
    v; a fixed point of the relaxed sweep is a fixed point of Eq. iteration.

    translate (an extension, not in the paper): before each half-sweep, the
    ``translation_step`` between the side just updated (the partner of the
    half-sweep) and the side about to be updated: before the u step,
    log v + tau, log u - tau; before the v step, log u + tau', log v - tau'.
    Each step maximises the same concave dual as the half-sweeps, so the
    fixed point is that of Eq. iteration. With tol, the residual is that of
    the state after the first translation (the state the u step starts from).

    Returns a dict: log_u, log_v, sweeps (number of sweeps run), res_inf,
    res_l1 (of the returned state) and trace (res_inf before each sweep when
    tol is given).
    """
    logA = log_kernel(Phi, beta)
    N, M = logA.shape
    lu = np.zeros(N) if log_u is None else np.array(log_u, dtype=np.float64)
    lv = np.zeros(M) if log_v is None else np.array(log_v, dtype=np.float64)
    trace = []
    sweeps = 0
    for _ in range(int(max_sweeps)):
        if translate:
            lv, lu, _ = translation_step(lv, lu, m, n)
        if tol is not None:
            r_inf, _, _ = row_residual(logA, n, lu, lv)
            trace.append(r_inf)
            if r_inf <= tol:
                break
        if omega == 1.0:
            lu = half_sweep_x(logA, lv, n)
        else:
            lu = lu + omega * (half_sweep_x(logA, lv, n) - lu)
        if translate:
            lu, lv, _ = translation_step(lu, lv, n, m)
        if omega == 1.0:
            lv = half_sweep_y(logA, lu, m)
        else:
            lv = lv + omega * (half_sweep_y(logA, lu, m) - lv)
        sweeps += 1
    r_inf, r_l1, _ = row_residual(logA, n, lu, lv)
    return dict(log_u=lu, log_v=lv, sweeps=sweeps, res_inf=r_inf, res_l1=r_l1, trace=trace)


def ipfp_jacobi(Phi, n, m, beta, max_sweeps, tol=None, log_u=None, log_v=None):
    """The Jacobi variant of Eq. iteration (an extension, not in the paper):
    both half-sweeps of a sweep read the state entering it, u' from the old v
    and v' from the old u, so one pass over the pairs could feed both. Same
    fixed point (Eq. IPFP). With tol, the loop stops before a sweep whose
    entering state has row residual <= tol. Returns a dict like ipfp_batch,
    with states: the (log u, log v) after every sweep."""
    logA = log_kernel(Phi, beta)
    N, M = logA.shape
    lu = np.zeros(N) if log_u is None else np.array(log_u, dtype=np.float64)
    lv = np.zeros(M) if log_v is None else np.array(log_v, dtype=np.float64)
    trace, states = [], []
    sweeps = 0
    for _ in range(int(max_sweeps)):
        if tol is not None:
            r_inf, _, _ = row_residual(logA, n, lu, lv)
            trace.append(r_inf)
            if r_inf <= tol:
                break
        lu, lv = half_sweep_x(logA, lv, n), half_sweep_y(logA, lu, m)
        states.append((lu, lv))
        sweeps += 1
    r_inf, r_l1, _ = row_residual(logA, n, lu, lv)
    return dict(log_u=lu, log_v=lv, sweeps=sweeps, res_inf=r_inf, res_l1=r_l1, trace=trace, states=states)


def ipfp_batch_literal(P, Q, n, m, beta, iters):
    """Alg. 1 exactly as printed, in the linear domain and with the printed
    update sqrt(s^2 + n) - s. Only for small, well-conditioned markets (it
    overflows and cancels where the log form does not). Returns (u, v, mu)."""
    A = np.exp((np.asarray(P, np.float64) + np.asarray(Q, np.float64)) / (2.0 * beta))
    u = np.ones(A.shape[0])
    v = np.ones(A.shape[1])
    for _ in range(int(iters)):
        s = A @ v / 2.0
        u = np.sqrt(s ** 2 + n) - s
        s = A.T @ u / 2.0
        v = np.sqrt(s ** 2 + m) - s
    mu = A * np.outer(u, v)
    return u, v, mu


# ---------------------------------------------------------------------------
# Mini-batch IPFP (Alg. 2)
# ---------------------------------------------------------------------------

def ipfp_minibatch(F, K, G, L, n, m, beta, sweeps, rows_per_batch_x, rows_per_batch_y,
                   bias_x=None, bias_y=None, log_u=None, log_v=None):
    """Mini-batch IPFP, Alg. 2 / Eq. iteration_minibatch, in logs.

    The X users are cut into consecutive batches of ``rows_per_batch_x`` rows
    (the last one ragged), the Y users likewise. For batch j of X:
    A_j = exp((F_j G^T + K_j L^T) / (2 beta)) (size B x |Y|), s_j = A_j v / 2,
    u_j = sqrt(n_j + s_j^2) - s_j; then for batch j of Y:
    (A^T)_j = exp((G_j F^T + L_j K^T) / (2 beta)) (size B x |X|), s_j = (A^T)_j u / 2,
    v_j = sqrt(m_j + s_j^2) - s_j. Phi is never formed whole.

    Returns a dict: log_u, log_v, Psi, Xi (``stable_factors`` of the result).
    """
    F = np.asarray(F, np.float64); K = np.asarray(K, np.float64)
    G = np.asarray(G, np.float64); L = np.asarray(L, np.float64)
    N, M = F.shape[0], G.shape[0]
    bx = np.zeros(N) if bias_x is None else np.asarray(bias_x, np.float64)
    by = np.zeros(M) if bias_y is None else np.asarray(bias_y, np.float64)
    lu = np.zeros(N) if log_u is None else np.array(log_u, dtype=np.float64)
    lv = np.zeros(M) if log_v is None else np.array(log_v, dtype=np.float64)
    for _ in range(int(sweeps)):
        for j0 in range(0, N, rows_per_batch_x):
            j1 = min(N, j0 + rows_per_batch_x)
            logA_j = (F[j0:j1] @ G.T + K[j0:j1] @ L.T + bx[j0:j1, None] + by[None, :]) / (2.0 * beta)
            log_s = LOG_HALF + _logsumexp(logA_j + lv[None, :], axis=1)
            lu[j0:j1] = scaling_update(log_s, n[j0:j1])
        for j0 in range(0, M, rows_per_batch_y):
            j1 = min(M, j0 + rows_per_batch_y)
            logAT_j = (G[j0:j1] @ F.T + L[j0:j1] @ K.T + by[j0:j1, None] + bx[None, :]) / (2.0 * beta)
            log_s = LOG_HALF + _logsumexp(logAT_j + lu[None, :], axis=1)
            lv[j0:j1] = scaling_update(log_s, m[j0:j1])
    Psi, Xi = stable_factors(F, K, G, L, beta, lu, lv, bias_x, bias_y)
    return dict(log_u=lu, log_v=lv, Psi=Psi, Xi=Xi)


# ---------------------------------------------------------------------------
# Outputs: mu, match count, stable factors, welfare, ranked lists
# ---------------------------------------------------------------------------

def log_mu(logA, log_u, log_v):
    """Eq. stable_condition with u = sqrt(mu_x0), v = sqrt(mu_0y):
    mu_xy = A_xy u_x v_y (Alg. 1, final line mu = A (.) (u (x) v)), as log mu."""
    return logA + np.asarray(log_u)[:, None] + np.asarray(log_v)[None, :]


def match_count(n, log_u, m=None, log_v=None):
    """Total matched mass sum_xy mu_xy.

    From the row equations of Eq. IPFP, sum_y mu_xy = n_x - mu_x0 = n_x - u_x^2, so
    sum_xy mu_xy = sum n - sum u^2 (and = sum m - sum v^2 from the columns).
    Returns the X-side form, or both forms when m and log_v are given.
    """
    cx = float(np.sum(n) - np.sum(np.exp(2.0 * np.asarray(log_u))))
    if m is None:
        return cx
    cy = float(np.sum(m) - np.sum(np.exp(2.0 * np.asarray(log_v))))
    return cx, cy


def stable_factors(F, K, G, L, beta, log_u, log_v, bias_x=None, bias_y=None):
    """Stable factor matrices Psi (N x (2D+2)) and Xi (M x (2D+2)) of Alg. 2
    (final lines) and the Tomita et al. embedding of Sec. 3.3, with
    log mu_xy = <psi_x, xi_y> / (2 beta).

    Reading: as printed, psi carries beta log u and xi carries beta log v; then
    <psi, xi>/(2 beta) = phi/(2 beta) + (log u + log v)/2, which contradicts
    Eq. stable_condition. The entries must be 2 beta log u and 2 beta log v,
    which makes the inner product exactly phi/(2 beta) + log u + log v. With
    popularity biases, b_x and b_y are added to those two entries.
    """
    F = np.asarray(F, np.float64); K = np.asarray(K, np.float64)
    G = np.asarray(G, np.float64); L = np.asarray(L, np.float64)
    N, M = F.shape[0], G.shape[0]
    bx = np.zeros(N) if bias_x is None else np.asarray(bias_x, np.float64)
    by = np.zeros(M) if bias_y is None else np.asarray(bias_y, np.float64)
    Psi = np.concatenate([F, K, (2.0 * beta * np.asarray(log_u) + bx)[:, None], np.ones((N, 1))], axis=1)
    Xi = np.concatenate([G, L, np.ones((M, 1)), (2.0 * beta * np.asarray(log_v) + by)[:, None]], axis=1)
    return Psi, Xi


def welfare(Phi, mu, n, m, beta):
    """Social welfare objective of Eq. primary optimization evaluated at mu:
        sum_xy mu_xy phi_xy + beta E(mu),
        E(mu) = -sum_{x, y in Y0} mu_xy log(mu_xy / n_x) - sum_{y, x in X0} mu_xy log(mu_xy / m_y),
    with the unmatched masses mu_x0 = n_x - sum_y mu_xy, mu_0y = m_y - sum_x mu_xy
    taken from the constraints. Returns -inf outside the feasible set."""
    mu = np.asarray(mu, np.float64)
    n = np.asarray(n, np.float64); m = np.asarray(m, np.float64)
    mu_x0 = n - mu.sum(axis=1)
    mu_0y = m - mu.sum(axis=0)
    if np.any(mu <= 0) or np.any(mu_x0 <= 0) or np.any(mu_0y <= 0):
        return -np.inf
    e_x = -np.sum(mu * np.log(mu / n[:, None])) - np.sum(mu_x0 * np.log(mu_x0 / n))
    e_y = -np.sum(mu * np.log(mu / m[None, :])) - np.sum(mu_0y * np.log(mu_0y / m))
    return float(np.sum(mu * Phi) + beta * (e_x + e_y))


def topk_partners(logA, log_u, log_v, k, side=0):
    """Ranked recommendation lists: for each user of ``side`` (0: X users rank
    Y partners, 1: Y users rank X partners), the k partners with the largest
    mu_xy (Eq. stable_condition), largest first.

    Reading (the paper ranks lists per user, Sec. 4.1, without a tie rule): equal
    scores are ordered by lower partner index. Returns (idx int64, log mu).
    """
    lm = log_mu(logA, log_u, log_v)
    if side == 1:
        lm = lm.T
    k = int(min(k, lm.shape[1]))
    order = np.argsort(-lm, axis=1, kind="stable")[:, :k]
    vals = np.take_along_axis(lm, order, axis=1)
    return order.astype(np.int64), vals


# ---------------------------------------------------------------------------
# Sampled certification for markets too large to solve on the CPU
# ---------------------------------------------------------------------------

def sampled_row_update(F, K, G, L, beta, mass, log_v, rows, bias_x=None, bias_y=None,
                       col_chunk=65536):
    """One X half-sweep (Eq. iteration_minibatch, first line) restricted to the
    given rows: the mini-batch A_j is formed for those rows only, in column
    chunks, and the rows' new log u is returned together with log s.

    The same function with the sides exchanged (G, L, F, K, bias_y, bias_x and
    the Y capacities) gives the Y half-sweep for sampled columns.
    Returns (log_s, log_u_new) for ``rows``.
    """
    rows = np.asarray(rows, dtype=np.int64)
    Fj = np.asarray(F[rows], np.float64)
    Kj = np.asarray(K[rows], np.float64)
    bxj = np.zeros(len(rows)) if bias_x is None else np.asarray(bias_x, np.float64)[rows]
    M = G.shape[0]
    # running log-sum-exp over column chunks (a partition of the sum over y)
    run_max = np.full(len(rows), -np.inf)
    run_sum = np.zeros(len(rows))
    for c0 in range(0, M, col_chunk):
        c1 = min(M, c0 + col_chunk)
        Gc = np.asarray(G[c0:c1], np.float64)
        Lc = np.asarray(L[c0:c1], np.float64)
        byc = np.zeros(c1 - c0) if bias_y is None else np.asarray(bias_y[c0:c1], np.float64)
        a = (Fj @ Gc.T + Kj @ Lc.T + bxj[:, None] + byc[None, :]) / (2.0 * beta)
        a = a + np.asarray(log_v[c0:c1], np.float64)[None, :]
        cm = np.max(a, axis=1)
        new_max = np.maximum(run_max, cm)
        run_sum = run_sum * np.exp(run_max - new_max) + np.sum(np.exp(a - new_max[:, None]), axis=1)
        run_max = new_max
    log_s = LOG_HALF + run_max + np.log(run_sum)
    return log_s, scaling_update(log_s, np.asarray(mass, np.float64)[rows])


# ---------------------------------------------------------------------------
# Expected number of matches of ranked lists (Sec. 4.1)
# ---------------------------------------------------------------------------

def expected_matches(P, Q, lists_x, lists_y):
    """Expected matches of the ranked lists shown to both sides, under the
    position-based model with examination v(k) = 1 / exp(k - 1) (Sec. 4.1).
    Reading (the paper takes the measure from Su et al. without restating it):
    x and y match when each examines and likes the other, so the expectation
    is the sum over all pairs of v(pos_x(y)) P[x, y] v(pos_y(x)) Q[y, x], with
    v = 0 for a partner missing from a list. lists_x[x] is the sequence of y's
    shown to x (best first), lists_y[y] that of x's shown to y. A plain double
    loop over the pairs."""
    N, M = len(lists_x), len(lists_y)
    total = 0.0
    for x in range(N):
        for y in range(M):
            lx = list(lists_x[x])
            ly = list(lists_y[y])
            if y in lx and x in ly:
                kx = lx.index(y) + 1
                ky = ly.index(x) + 1
                total += np.exp(-(kx - 1)) * P[x][y] * np.exp(-(ky - 1)) * Q[y][x]
    return float(total)
