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


def _market():
    return make_market(37, 53, 4, sigma=0.7, seed=5, bias_x=True, bias_y=True, n_kind="uniform_real",
                       m_kind="uniform_real", dtype="fp32")


def _worker(rank, world, port, q, translate):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mk = _market()
        f = mk.f64()
        Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"])
        logA = oracle.log_kernel(Phi, f["sigma"])

        def half_x_res(lo, hi, log_u, log_v):
            lv = log_v.numpy()
            _, _, r = oracle.row_residual(logA[lo:hi], f["n"][lo:hi], log_u.numpy()[lo:hi], lv)
            new = oracle.half_sweep_x(logA[lo:hi], lv, f["n"][lo:hi])
            return torch.from_numpy(new), float(np.max(np.abs(r) / f["n"][lo:hi])) if hi > lo else 0.0

        def half_y(lo, hi, log_u, log_v):
            new = oracle.half_sweep_y(logA[:, lo:hi], log_u.numpy(), f["m"][lo:hi])
            return torch.from_numpy(new), 0.0

        lu = torch.zeros(mk.N, dtype=torch.float64)
        lv = torch.zeros(mk.M, dtype=torch.float64)
        lu, lv, res = sharded_sweeps(half_x_res, half_y, lu, lv, 6, translate=translate,
                                     n_sum=float(np.sum(f["n"])), m_sum=float(np.sum(f["m"])))
        if rank == 0:
            q.put((lu.numpy(), lv.numpy(), res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("translate", [False, True], ids=["plain", "translated"])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_iterates_equal_oracle(world, translate):
    """The sharded schedule's iterates after 6 sweeps are the oracle's unsharded
    ones (with and without the translation step, taken on the host from the
    gathered vectors), and its MAX-reduced residual is the oracle's residual of
    the state entering the 6th sweep's u step."""
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, translate)) for r in range(world)]
    for p in procs:
        p.start()
    lu, lv, res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f = _market().f64()
    Phi = oracle.phi_dense(f["F"], f["K"], f["G"], f["L"], f["bias_x"], f["bias_y"])
    ref5 = oracle.ipfp_batch(Phi, f["n"], f["m"], f["sigma"], max_sweeps=5, translate=translate)
    ref6 = oracle.ipfp_batch(Phi, f["n"], f["m"], f["sigma"], max_sweeps=6, translate=translate)
    np.testing.assert_allclose(lu, ref6["log_u"], atol=1e-12)
    np.testing.assert_allclose(lv, ref6["log_v"], atol=1e-12)
    lu5, lv5 = ref5["log_u"], ref5["log_v"]
    if translate:
        lv5, lu5, _ = oracle.translation_step(lv5, lu5, f["m"], f["n"])
    r5, _, _ = oracle.row_residual(oracle.log_kernel(Phi, f["sigma"]), f["n"], lu5, lv5)
    assert res == pytest.approx(r5, rel=1e-9)


def test_host_translation_tau_is_the_oracles():
    """The sharded schedule's host-side translation step (the product's own
    closed form) gives the oracle's tau, for both signs of the capacity
    difference and for potentials whose squares overflow float64."""
    from paper_2411_19214_gb300.sharded import translation_tau
    rng = np.random.default_rng(3)
    for cp, co, dm in [(0.0, 0.0, 0.0), (150.0, -200.0, 3.0), (-300.0, 250.0, -2.0), (5.0, 4.0, -7.5)]:
        lp = cp + rng.normal(0.0, 1.0, 6)
        lo = co + rng.normal(0.0, 1.0, 5)
        mass_o = rng.uniform(0.5, 2.0, 5)
        mass_p = np.full(6, (np.sum(mass_o) + dm) / 6.0)
        _, _, want = oracle.translation_step(lp, lo, mass_p, mass_o)
        got = translation_tau(lp, lo, float(np.sum(mass_p)), float(np.sum(mass_o)))
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (got, want)


def test_shard_ranges_cover_exactly():
    for n in (1, 2, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard_range(n, world, r)
                assert 0 <= lo <= hi <= n
                seen.extend(range(lo, hi))
            assert seen == list(range(n))
