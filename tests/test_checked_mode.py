"""Checked mode (guard bands around every market buffer, verified when the
buffer is freed) changes no result and finds no out-of-bounds writes on the
fused and dense paths: sweeps, the ranked lists (both list kinds), mu blocks,
a solve, potentials in and out, a factor update and a ranking-stop solve."""

import numpy as np
import pytest
import torch

from synth import make_market

pytestmark = pytest.mark.gpu


def _dev(a, path):
    """Factors in the market's element type (bf16 bit patterns on the fused path, float32 on the dense one)."""
    if path == "fused":
        bits = (np.ascontiguousarray(a, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)
        return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _exercise(tu, mk, path):
    mkt = tu.from_synth(mk, path=path)
    try:
        out = {}
        mkt.sweep(3)
        out["pot3"] = [t.cpu().numpy() for t in mkt.potentials()]
        for k in (10, 20):
            idx, lm = mkt.topk(0, k)
            out[f"topk{k}"] = (idx.cpu().numpy(), lm.cpu().numpy())
            idx, lm = mkt.topk(1, k)
            out[f"topkY{k}"] = (idx.cpu().numpy(), lm.cpu().numpy())
        out["mu"] = mkt.mu_block(0, 40, 3, 200).cpu().numpy()
        info = mkt.solve(tol=1e-5, max_iter=3000)
        out["solve"] = (info["sweeps"], info["residual_inf"])
        lu, lv = mkt.potentials()
        mkt.set_potentials(lu, lv)
        mkt.update_factors(*(_dev(a, path) for a in (mk.F, mk.K, mk.G, mk.L)))
        mkt.sweep(2)
        out["pot_after"] = [t.cpu().numpy() for t in mkt.potentials()]
        rinfo = mkt.solve_ranking(k=5, sample=64, check_every=4, patience=2, max_iter=400)
        out["rank"] = rinfo["sweeps"]
        return out
    finally:
        mkt.close()


@pytest.mark.parametrize("path", ["fused", "dense"])
def test_checked_mode_same_results_no_violations(gpu_lib, path):
    tu = gpu_lib
    mk = make_market(700, 1333, 24, sigma=0.5, seed=77, bias_x=True, bias_y=True, n_kind="uniform1to3",
                     m_kind="uniform1to3", dtype="bf16" if path == "fused" else "fp32")
    before, _ = tu.tu_guard_violations()
    tu.tu_set_checked_mode(False)
    plain = _exercise(tu, mk, path)
    tu.tu_set_checked_mode(True)
    try:
        checked = _exercise(tu, mk, path)
        torch.cuda.synchronize()
    finally:
        import os
        tu.tu_set_checked_mode(os.environ.get("TU_CHECKED") == "1")
    n, last = tu.tu_guard_violations()
    assert n == before, last
    assert plain.keys() == checked.keys()
    for key in plain:
        a, b = plain[key], checked[key]
        if isinstance(a, (list, tuple)):
            for x, y in zip(a, b):
                np.testing.assert_array_equal(np.asarray(x), np.asarray(y), err_msg=key)
        else:
            np.testing.assert_array_equal(np.asarray(a), np.asarray(b), err_msg=key)
