"""Expected number of matches of ranked recommendation lists (Sec. 4.1).

Sec. 4.1 evaluates the lists a matching policy shows to both sides by the
expected number of matches under a position-based model whose examination
function is v(k) = 1 / exp(k - 1), k the 1-based position in a list. Reading
(the paper takes the measure from Su et al. 2022 without restating it): a
match between candidate x and employer y needs both to examine and like each
other, so

    E[matches] = sum_{x, y} v(pos_x(y)) P_xy v(pos_y(x)) Q_yx,

where pos_x(y) is y's position in x's list (v = 0 when y is not in it) and
P_xy, Q_yx are the probabilities that x likes y and y likes x. The lists
here are the library's ranked lists (tu_topk_partners on both sides); for k
of 20 or more the positions left out carry v < 3e-9. Host code over the
k-entry lists: O((N + M) k).
"""

from __future__ import annotations

import numpy as np


def examination(pos) -> np.ndarray:
    """v(k) = 1 / exp(k - 1) for 1-based positions k."""
    return np.exp(-(np.asarray(pos, np.float64) - 1.0))


def expected_matches(idx_x, idx_y, P, Q) -> float:
    """Expected matches of lists idx_x (N x k: the partners y of every
    candidate x, best first) and idx_y (M x k: the partners x of every
    employer y) under like-probabilities P (N x M) and Q (M x N)."""
    idx_x = np.asarray(idx_x, np.int64)
    idx_y = np.asarray(idx_y, np.int64)
    N, kx = idx_x.shape
    M, ky = idx_y.shape
    # (x, y, position) of every entry of both sides' lists, joined on the pair
    key_x = np.repeat(np.arange(N, dtype=np.int64), kx) * M + idx_x.ravel()
    key_y = idx_y.ravel() * M + np.repeat(np.arange(M, dtype=np.int64), ky)
    pos_x = np.tile(np.arange(1, kx + 1), N)
    pos_y = np.tile(np.arange(1, ky + 1), M)
    order = np.argsort(key_y, kind="stable")
    sk = key_y[order]
    at = np.searchsorted(sk, key_x)
    hit = (at < sk.size) & (sk[np.minimum(at, sk.size - 1)] == key_x)
    xs, ys = key_x[hit] // M, key_x[hit] % M
    vy = examination(pos_y[order][at[hit]])
    vx = examination(pos_x[hit])
    return float(np.sum(vx * vy * np.asarray(P, np.float64)[xs, ys] * np.asarray(Q, np.float64)[ys, xs]))
