"""Write closed_forms.json: exact equilibria of markets small enough to solve by hand.

Uses only mpmath (50 significant digits); it does not call the oracle or the
CUDA path.

1x1 market (Eq. stable_condition and Eq. IPFP with one user per side): with
a = exp(phi / (2 beta)), mu = a u v, u^2 = n - mu and v^2 = m - mu, so
mu^2 = a^2 (n - mu)(m - mu), i.e. (a^2 - 1) mu^2 - a^2 (n + m) mu + a^2 n m = 0;
the equilibrium is the root in (0, min(n, m)). For a = 1 it is n m / (n + m).

Symmetric 2x2 market with unit capacities and phi = [[alpha, gamma], [gamma, alpha]]:
by symmetry u1 = u2 = v1 = v2 = w, and the row equation of Eq. IPFP reads
w^2 + w (e^{alpha/2beta} + e^{gamma/2beta}) w = 1, so w = 1 / sqrt(1 + e^{alpha/2beta} + e^{gamma/2beta}).
"""
import json
import os

import mpmath as mp

mp.mp.dps = 50


def mu_1x1(phi, beta, n, m):
    phi, beta, n, m = (mp.mpf(str(t)) for t in (phi, beta, n, m))
    a2 = mp.e ** (phi / beta)          # a^2 = exp(phi / beta)
    if a2 == 1:
        return n * m / (n + m)
    A, B, C = a2 - 1, -a2 * (n + m), a2 * n * m
    disc = mp.sqrt(B * B - 4 * A * C)
    roots = [(-B - disc) / (2 * A), (-B + disc) / (2 * A)]
    good = [r for r in roots if 0 < r < min(n, m)]
    assert len(good) == 1, roots
    return good[0]


def w_2x2(alpha, gamma, beta):
    alpha, gamma, beta = (mp.mpf(str(t)) for t in (alpha, gamma, beta))
    return 1 / mp.sqrt(1 + mp.e ** (alpha / (2 * beta)) + mp.e ** (gamma / (2 * beta)))


def main():
    cases_1x1 = [
        dict(phi=0.0, beta=1.0, n=1.0, m=1.0),
        dict(phi=1.3, beta=0.5, n=1.0, m=2.0),
        dict(phi=-2.0, beta=1.0, n=0.3, m=0.7),
        dict(phi=6.0, beta=0.5, n=1.0, m=1.0),
        dict(phi=-30.0, beta=1.0, n=5.0, m=2.0),
        dict(phi=3.0, beta=2.0, n=1e-6, m=1e-6),
    ]
    for c in cases_1x1:
        c["mu"] = mp.nstr(mu_1x1(c["phi"], c["beta"], c["n"], c["m"]), 30)
    cases_2x2 = [
        dict(alpha=0.7, gamma=-0.4, beta=1.0),
        dict(alpha=-1.5, gamma=2.5, beta=0.5),
    ]
    for c in cases_2x2:
        c["w"] = mp.nstr(w_2x2(c["alpha"], c["gamma"], c["beta"]), 30)
    out = dict(
        description="Exact equilibria of 1x1 and symmetric 2x2 markets (closed forms in make_closed_forms.py).",
        citation="Eq. stable_condition and Eq. IPFP (Sec. 3.2); 1x1: mu = a u v with u^2 = n - mu, v^2 = m - mu.",
        one_by_one=cases_1x1,
        symmetric_two_by_two=cases_2x2,
    )
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
