"""CPU float64 oracle for the Choo-Siow / Galichon-Salanie IPFP.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct
restatement of what the paper computes, used to check the CUDA path. Only the
tests, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and
its reference arm) may import it. The product package
``paper_2411_19214_gb300`` never imports it, and it imports nothing from the
product package: the two share no code.

Every function cites the passage of the paper it follows (section, equation
label or algorithm). Where the paper is silent or garbled, the reading taken is
stated in the function's docstring.

Pins (in ``tests/test_oracle.py``, all run on the CPU):

* closed-form 1x1 market (quadratic in mu) and symmetric 2x2 market;
* Newton's method on the concave dual, independent of the IPFP iteration;
* direct maximisation of the social-welfare primal (Eq. primary optimization),
  which pins the 2*beta in the kernel;
* the literal Alg. 1 update (printed form) on well-conditioned markets;
* invariants at the fixed point (marginals, total mass identity, permutation
  equivariance, side swap, mass scaling) and batch == mini-batch iterates;
* brute-force sorting for the ranked lists;
* the translation step (an extension) against a brute-force maximisation of
  the dual along its line and a 60-digit root of its quadratic;
* the Jacobi order (an extension) against Gauss-Seidel: its iterates are two
  interleaved Gauss-Seidel sequences.
"""

from .ipfp import (  # noqa: F401
    phi_dense,
    log_kernel,
    asinh_exp,
    scaling_update,
    half_sweep_x,
    half_sweep_y,
    ipfp_batch,
    ipfp_jacobi,
    dual_value,
    translation_step,
    ipfp_batch_literal,
    ipfp_minibatch,
    row_residual,
    col_residual,
    log_mu,
    match_count,
    stable_factors,
    welfare,
    topk_partners,
    sampled_row_update,
    expected_matches,
)
