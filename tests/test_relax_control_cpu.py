"""The relaxation controller of the solve loops, on given residual traces.

tu_relax_schedule runs the host-side controller tu_ipfp_solve uses (no CUDA
call), so its policy is checked here on the CPU: plain sweeps until a decay
rate is measured below a residual of 0.1; then a fixed factor is applied as
set all the way down to tol, while the automatic factor
2 / (1 + sqrt(1 - q)) is lowered linearly towards 1 over the last decade of
the residual above tol; a tenfold rise over the best residual halves the
factor's excess over 1.
"""

import numpy as np
import pytest

import paper_2411_19214_gb300 as tu
from paper_2411_19214_gb300 import build as tb


@pytest.fixture(scope="module", autouse=True)
def _lib():
    tb.build()
    tu.load()


def _trace(q=0.99, r0=0.05, block=16, blocks=40):
    done = np.arange(1, blocks + 1) * block
    return done, r0 * q ** done


def test_fixed_factor_is_applied_down_to_tol():
    done, r = _trace()
    tol = r[-1] / 3.0  # the last observations lie within a decade of tol
    om = tu.tu_relax_schedule(1.5, tol, done, r)
    first = int(np.argmax(om > 1.0))
    assert 0 < first <= 3, om[:5]  # plain until a rate is measured
    assert np.all(om[:first] == 1.0)
    assert np.all(om[first:] == 1.5), om
    assert np.any(r[first:] < 10 * tol)  # the check covers the last decade


def test_automatic_factor_tapers_over_the_last_decade():
    q = 0.99
    done, r = _trace(q=q)
    tol = r[-1] / 3.0
    om = tu.tu_relax_schedule(0.0, tol, done, r)
    target = min(1.98, 2.0 / (1.0 + np.sqrt(1.0 - q)))
    far = r > 10 * tol
    active = om > 1.0
    # away from tol the controller applies the successive over-relaxation factor
    assert np.any(far & active)
    np.testing.assert_allclose(om[far & active], target, rtol=1e-6)
    # within the last decade it interpolates linearly in log10(r / tol)
    near = (~far) & (np.arange(len(r)) > int(np.argmax(active)))
    assert np.any(near)
    want = 1.0 + (target - 1.0) * np.log10(r[near] / tol)
    np.testing.assert_allclose(om[near], want, atol=1.1e-3)


def test_tenfold_rise_halves_the_excess():
    done, r = _trace()
    tol = 1e-12
    r = r.copy()
    k = 10
    r[k:] = r[k:] * 20.0  # a sudden rise over the best residual seen
    om = tu.tu_relax_schedule(1.8, tol, done, r)
    assert om[k - 1] == pytest.approx(1.8)
    assert om[k] == pytest.approx(1.4)
    assert np.all(om[k:] == pytest.approx(1.4))


def test_invalid_schedules_rejected():
    done, r = _trace(blocks=3)
    for args in [(0.5, 1e-6, done, r), (2.0, 1e-6, done, r), (1.5, -1.0, done, r),
                 (1.5, 1e-6, np.array([16, 16, 32]), r), (1.5, 1e-6, np.array([0, 16, 32]), r)]:
        with pytest.raises(tu.TuError) as e:
            tu.tu_relax_schedule(*args)
        assert e.value.status == tu.TU_ERR_INVALID_ARG
