"""One market split into shards on the library's row-range half-sweep (GPU).

A rank of a market split across GPUs updates only its contiguous shard of a
side against the other side's full potentials (Sec. 3.3, Eq. iteration:
within a half-sweep each user depends only on the other side). Here (one GPU
available) the shards are checked two ways: in one process, shards of a side
computed one after another reproduce the whole-side half-sweep bit for bit;
and the sharded schedule (paper_2411_19214_gb300.sharded) runs as two gloo
ranks, each with its own copy of the market on the one GPU, the all-gathers
and the translation step on the host, against the oracle's translated
iterates. The two processes' kernels never wait on one another.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

from synth import make_market

from _parity import oracle_sweeps

pytestmark = pytest.mark.gpu

ATOL_LOG = 2e-5


def _mk():
    return make_market(1030, 777, 32, sigma=0.5, seed=91, bias_x=True, bias_y=True, n_kind="uniform_real",
                       m_kind="uniform_real", dtype="bf16")


@pytest.mark.parametrize("cuts", [[0, 300, 1030], [0, 1, 257, 1029, 1030], [0, 0, 1030]])
def test_shards_reproduce_the_whole_half_sweep(gpu_lib, cuts):
    """Shards [c_i, c_{i+1}) of X (then of Y), each a range half-sweep from the
    same state, give the whole side's half-sweep bit for bit; their residual
    maxima combine to the whole pass's, and ragged, one-user and empty shards
    work."""
    tu = gpu_lib
    mk = _mk()
    whole = tu.from_synth(mk)
    part = tu.from_synth(mk)
    try:
        whole.set_translation(False)
        whole.sweep(2)
        lu0, lv0 = whole.potentials64()
        tu.tu_set_potentials_f64(part.handle, lu0, lv0)
        res_whole = whole.sweep(0, residual=True)
        whole.sweep(1)  # the u step, then the v step from the new u
        wu, wv = whole.potentials64()
        res_max = 0.0
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            r = tu.tu_ipfp_half_sweep_range(part.handle, 0, lo, hi, residual=True)
            res_max = max(res_max, r[0])
        pu, _ = part.potentials64()
        np.testing.assert_array_equal(pu, wu)
        assert res_max == res_whole
        ycuts = [min(c, mk.M) for c in cuts[:-1]] + [mk.M]
        for lo, hi in zip(ycuts[:-1], ycuts[1:]):
            tu.tu_ipfp_half_sweep_range(part.handle, 1, lo, hi)
        _, pv = part.potentials64()
        np.testing.assert_array_equal(pv, wv)
        shard = np.empty(5)
        tu.tu_get_potentials_range_f64(part.handle, 1, 3, 8, shard)
        np.testing.assert_array_equal(shard, pv[3:8])
        for bad in [(0, -1, 5), (0, 5, 4), (0, 0, mk.N + 1), (2, 0, 1)]:
            with pytest.raises(tu.TuError) as e:
                tu.tu_ipfp_half_sweep_range(part.handle, *bad)
            assert e.value.status == tu.TU_ERR_INVALID_ARG
    finally:
        whole.close()
        part.close()


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
        import paper_2411_19214_gb300 as tu
        from paper_2411_19214_gb300.sharded import library_half_sweeps, sharded_sweeps
        torch.cuda.set_device(0)
        tu.load()
        mk = _mk()
        mkt = tu.from_synth(mk)
        try:
            hx, hy = library_half_sweeps(mkt.handle)
            lu = torch.zeros(mk.N, dtype=torch.float64)
            lv = torch.zeros(mk.M, dtype=torch.float64)
            lu, lv, res = sharded_sweeps(hx, hy, lu, lv, 4, translate=True, n_sum=float(np.sum(mk.n)),
                                         m_sum=float(np.sum(mk.m)))
        finally:
            mkt.close()
        if rank == 0:
            q.put((lu.numpy(), lv.numpy(), res))
    finally:
        dist.destroy_process_group()


def test_sharded_schedule_on_the_library_matches_the_oracle(gpu_lib):
    """Two gloo ranks, each a copy of the market on the GPU updating its shard
    through the row-range entry points; after 4 translated sweeps the gathered
    potentials are the oracle's translated iterates."""
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    lu, lv, res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ou, ov = oracle_sweeps(_mk(), 4, translate=True)
    np.testing.assert_allclose(lu, ou, rtol=0, atol=ATOL_LOG)
    np.testing.assert_allclose(lv, ov, rtol=0, atol=ATOL_LOG)
    assert np.isfinite(res) and res > 0.0
