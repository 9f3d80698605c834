"""Partner split and the launch-shape autotuner (GPU).

A split half-sweep cuts each own tile's partner tiles into ranges handled by
different CTAs; the warp that completes a tile's block of rows sums the
ranges' partial sums in range order. The iterates must match the oracle like
the unsplit ones (ATOL_LOG, derived in test_parity_fused.py), with every
tile-height mode, ragged tails, more ranges than partner tiles, graph replay
(the arrival counters reset themselves) and the reported residual. The
autotuner must leave the potentials untouched, keep a shape that is among its
candidates, and hand its choice to a later market of the same shape.
"""

import numpy as np
import pytest
import torch

import oracle
from synth import make_market

from _parity import dense_logA, oracle_sweeps

pytestmark = pytest.mark.gpu

ATOL_LOG = 2e-5


def _mk(N, M, d=32, seed=0):
    return make_market(N, M, d, sigma=0.5, seed=seed, bias_x=True, bias_y=True, n_kind="uniform_real",
                       m_kind="uniform_real", dtype="bf16")


@pytest.mark.parametrize("N,M,split,mode", [(3000, 2100, 2, 0), (3000, 2100, 3, 1), (2049, 1100, 5, 2),
                                            (700, 100, 4, 0), (1, 900, 3, 0), (5000, 5000, 8, 0)],
                         ids=lambda v: str(v))
def test_split_sweeps_match_oracle(gpu_lib, N, M, split, mode):
    tu = gpu_lib
    mk = _mk(N, M, seed=N + M + split)
    mkt = tu.from_synth(mk)
    try:
        tu.tu_market_set_small_tiles(mkt.handle, mode)
        tu.tu_market_set_split(mkt.handle, split)
        assert tu.tu_market_get_shape(mkt.handle) == (mode, split)
        mkt.sweep(1)
        mkt.sweep(5)  # a captured graph of 5 sweeps: the counters must be back at 0 after every pass
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        ou, ov = oracle_sweeps(mk, 6)
        np.testing.assert_allclose(lu, ou, rtol=0, atol=ATOL_LOG)
        np.testing.assert_allclose(lv, ov, rtol=0, atol=ATOL_LOG)
        # the residual of the state (FP64 potentials), reduced from the combining warps
        res = mkt.sweep(0, residual=True)
        logA, f = dense_logA(mk)
        u64, v64 = mkt.potentials64()
        want, _, _ = oracle.row_residual(logA, f["n"], u64, v64)
        assert res == pytest.approx(want, rel=1e-3, abs=1e-7)
    finally:
        mkt.close()


def test_split_agrees_with_unsplit_to_rounding(gpu_lib):
    tu = gpu_lib
    mk = _mk(4000, 3000, seed=7)
    a, b = tu.from_synth(mk), tu.from_synth(mk)
    try:
        tu.tu_market_set_split(b.handle, 3)
        a.sweep(4)
        b.sweep(4)
        for x, y in zip(a.potentials(), b.potentials()):
            np.testing.assert_allclose(x.double().cpu().numpy(), y.double().cpu().numpy(), rtol=0, atol=2e-6)
    finally:
        a.close()
        b.close()


def test_autotune_keeps_state_and_caches_the_shape(gpu_lib, tmp_path):
    tu = gpu_lib
    tu.tu_autotune_cache_clear()
    mk = _mk(40_000, 40_000, d=64, seed=3)
    mkt = tu.from_synth(mk)
    other = None
    try:
        mkt.sweep(2)
        before = mkt.potentials64()
        info = tu.tu_market_autotune(mkt.handle, reps=2)
        after = mkt.potentials64()
        assert all(np.array_equal(x, y) for x, y in zip(before, after))
        assert info["candidates"] >= 3 and info["ms"] <= info["ms_default"] * 1.0001
        assert tu.tu_market_get_shape(mkt.handle) == (info["small_tiles"], info["split"])
        print(f"\nautotune 4e4 x 4e4 d=64: {info}")
        # the solve still reaches the oracle's iterates under the chosen shape
        mkt.sweep(1)
        # a new market of the same shape bucket starts with the tuned shape
        other = tu.from_synth(_mk(40_500, 39_800, d=64, seed=4))
        assert tu.tu_market_get_shape(other.handle) == (info["small_tiles"], info["split"])
        path = tmp_path / "tune.json"
        tu.tu_autotune_cache_save(str(path))
        tu.tu_autotune_cache_clear()
        third = tu.from_synth(_mk(40_000, 40_000, d=64, seed=5))
        assert tu.tu_market_get_shape(third.handle) == (1, 1)  # default without a cache entry
        third.close()
        tu.tu_autotune_cache_load(str(path))
        third = tu.from_synth(_mk(40_000, 40_000, d=64, seed=5))
        assert tu.tu_market_get_shape(third.handle) == (info["small_tiles"], info["split"])
        third.close()
    finally:
        mkt.close()
        if other is not None:
            other.close()
        tu.tu_autotune_cache_clear()


def test_shape_arguments(gpu_lib):
    tu = gpu_lib
    mk = _mk(300, 200, seed=9)
    mkt = tu.from_synth(mk)
    dense = tu.from_synth(mk, path="dense")
    try:
        for bad in (0, 9):
            with pytest.raises(tu.TuError) as e:
                tu.tu_market_set_split(mkt.handle, bad)
            assert e.value.status == tu.TU_ERR_INVALID_ARG
        with pytest.raises(tu.TuError) as e:
            tu.tu_market_set_small_tiles(mkt.handle, 3)
        assert e.value.status == tu.TU_ERR_INVALID_ARG
        with pytest.raises(tu.TuError) as e:
            tu.tu_market_autotune(mkt.handle, reps=0)
        assert e.value.status == tu.TU_ERR_INVALID_ARG
        for call in (lambda: tu.tu_market_set_split(dense.handle, 2), lambda: tu.tu_market_autotune(dense.handle)):
            with pytest.raises(tu.TuError) as e:
                call()
            assert e.value.status == tu.TU_ERR_UNSUPPORTED
    finally:
        mkt.close()
        dense.close()


@pytest.mark.parametrize("per,split,mode", [("rows", 3, 0), ("side", 2, 2), ("rows", 4, 2)])
def test_split_fp8_sweeps_match_oracle(gpu_lib, per, split, mode):
    """The split instantiations of the e4m3 kernels (per-row scales: the
    partner ranges carry their rows' scales; per-side: folded into c)."""
    from synth import fp8_quantized
    tu = gpu_lib
    mk = make_market(2100, 1500, 64, sigma=0.5, seed=split + len(per), bias_x=True, bias_y=True,
                     n_kind="uniform_real", m_kind="uniform_real", dtype="fp32")
    q, _ = fp8_quantized(mk, "row" if per == "rows" else "side")
    mkt = tu.from_synth(mk, fp8=per)
    try:
        tu.tu_market_set_small_tiles(mkt.handle, mode)
        tu.tu_market_set_split(mkt.handle, split)
        mkt.sweep(4)
        lu, lv = mkt.potentials64()
        ou, ov = oracle_sweeps(q, 4)
        np.testing.assert_allclose(lu, ou, rtol=0, atol=ATOL_LOG)
        np.testing.assert_allclose(lv, ov, rtol=0, atol=ATOL_LOG)
    finally:
        mkt.close()


@pytest.mark.parametrize("N,M,blocks,mode", [(3000, 2100, 3, 0), (2049, 1100, 4, 2), (700, 100, 3, 0),
                                             (5000, 5000, 2, 1)], ids=lambda v: str(v))
def test_partner_blocks_match_oracle(gpu_lib, N, M, blocks, mode):
    """Partner blocks: the split's partial sums with the items ordered block
    by block (all own tiles against block 0 first); iterates of captured
    sweeps against the oracle, and the shape reported as -blocks."""
    tu = gpu_lib
    mk = _mk(N, M, seed=N + M + 10 * blocks)
    mkt = tu.from_synth(mk)
    try:
        tu.tu_market_set_small_tiles(mkt.handle, mode)
        tu.tu_market_set_partner_blocks(mkt.handle, blocks)
        assert tu.tu_market_get_shape(mkt.handle) == (mode, -blocks)
        mkt.sweep(1)
        mkt.sweep(5)
        lu, lv = (t.double().cpu().numpy() for t in mkt.potentials())
        ou, ov = oracle_sweeps(mk, 6)
        np.testing.assert_allclose(lu, ou, rtol=0, atol=ATOL_LOG)
        np.testing.assert_allclose(lv, ov, rtol=0, atol=ATOL_LOG)
        tu.tu_market_set_split(mkt.handle, 2)  # a split replaces the blocks
        assert tu.tu_market_get_shape(mkt.handle) == (mode, 2)
        for bad in (0, 9):
            with pytest.raises(tu.TuError):
                tu.tu_market_set_partner_blocks(mkt.handle, bad)
    finally:
        mkt.close()
