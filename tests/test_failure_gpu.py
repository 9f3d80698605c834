"""Failure detection on the GPU without a fault: the bounded device-side wait
that every pipeline role of the tensor-core kernels uses is made to run out
(an mbarrier that nothing signals); the kernel reports the timeout through the
error word, returns, and the context stays usable."""

import time

import numpy as np
import pytest

from synth import make_market

pytestmark = pytest.mark.gpu


def test_device_wait_times_out_and_context_survives(gpu_lib):
    tu = gpu_lib
    t0 = time.perf_counter()
    st, waited = tu.tu_selftest_wait_timeout(0.25)
    wall = time.perf_counter() - t0
    assert st == tu.TU_ERR_TIMEOUT, tu.status_string(st)
    assert 0.25 <= waited < 1.0 and wall >= 0.25, (waited, wall)
    # the device still runs the solver normally afterwards
    mk = make_market(300, 500, 16, sigma=1.0, seed=3, dtype="bf16")
    mkt = tu.from_synth(mk)
    try:
        info = mkt.solve(tol=1e-6, max_iter=2000)
        assert info["converged"], info
    finally:
        mkt.close()
    for bad in (0.0, -1.0, 6.0):
        st, _ = tu.tu_selftest_wait_timeout(bad)
        assert st == tu.TU_ERR_INVALID_ARG
