"""The sharded single-market schedule on 2 and 3 CPU ranks (gloo).

Each rank updates a contiguous shard of X (then of Y) against the other side's
full potentials, with the oracle's float64 half-sweep restricted to the shard
as the per-shard computation; the iterates after several sweeps must equal the
oracle's unsharded batch iterates, and the MAX-reduced residual must equal the
oracle's residual of the entering state.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

import oracle
from paper_2411_19214_gb300.sharded import shard_range, sharded_sweeps
from synth import make_market


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mk = make_market(37, 53, 4, sigma=0.7, seed=5, bias_x=True, bias_y=True, n_kind="uniform_real",
                         m_kind="uniform_real", dtype="fp32")
        f = mk.f64()
        Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"])
        logA = oracle.log_kernel(Phi, f["sigma"])

        # log u of the state entering the X half-sweep (the last all-gathered one)
        state = {"lu": torch.zeros(mk.N, dtype=torch.float64)}

        def half_x_res(lo, hi, log_v):
            lv = log_v.numpy()
            lu_old = state["lu"].numpy()
            _, _, r = oracle.row_residual(logA[lo:hi], f["n"][lo:hi], lu_old[lo:hi], lv)
            new = oracle.half_sweep_x(logA[lo:hi], lv, f["n"][lo:hi])
            return torch.from_numpy(new), float(np.max(np.abs(r) / f["n"][lo:hi])) if hi > lo else 0.0

        def half_y(lo, hi, log_u):
            state["lu"] = log_u
            new = oracle.half_sweep_y(logA[:, lo:hi], log_u.numpy(), f["m"][lo:hi])
            return torch.from_numpy(new), 0.0

        lu = torch.zeros(mk.N, dtype=torch.float64)
        lv = torch.zeros(mk.M, dtype=torch.float64)
        lu, lv, res = sharded_sweeps(half_x_res, half_y, lu, lv, 6)
        if rank == 0:
            q.put((lu.numpy(), lv.numpy(), res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_iterates_equal_oracle(world):
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    lu, lv, res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mk = make_market(37, 53, 4, sigma=0.7, seed=5, bias_x=True, bias_y=True, n_kind="uniform_real",
                     m_kind="uniform_real", dtype="fp32")
    f = mk.f64()
    Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"])
    ref5 = oracle.ipfp_batch(Phi, f["n"], f["m"], f["sigma"], max_sweeps=5)
    ref6 = oracle.ipfp_batch(Phi, f["n"], f["m"], f["sigma"], max_sweeps=6)
    np.testing.assert_allclose(lu, ref6["log_u"], atol=1e-13)
    np.testing.assert_allclose(lv, ref6["log_v"], atol=1e-13)
    # residual of the state entering the 6th sweep = state after 5 sweeps
    assert res == pytest.approx(ref5["res_inf"], rel=1e-10)


def test_shard_ranges_cover_exactly():
    for n in (1, 2, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard_range(n, world, r)
                assert 0 <= lo <= hi <= n
                seen.extend(range(lo, hi))
            assert seen == list(range(n))
