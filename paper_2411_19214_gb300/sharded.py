"""Host schedule of one market's IPFP sweep sharded across ranks.

Within a half-sweep every user's update depends only on the other side's
fixed potentials (Eq. iteration), so the X users can be split into contiguous
shards, one per rank, each rank updating its shard against all of Y; the new
log u are then all-gathered before the Y half-sweep, which is split the same
way. The residual of the entering state (row equations of Eq. IPFP) is reduced
with a MAX all-reduce. Factors are replicated on every rank (0.5 GB at
1e6 x 1e6, d = 64). With ``translate`` the translation step (the exact
maximisation of the dual along log u + tau, log v - tau) precedes every
half-sweep, taken on the gathered vectors on the host, as the library takes it
for a whole market.

The per-shard half-sweep is passed in as a callable; :func:`library_half_sweeps`
makes the two callables of one GPU's market from the library's row-range
entry points.
"""

from __future__ import annotations

import math
from typing import Callable, Optional, Tuple

import numpy as np
import torch
import torch.distributed as dist


def shard_range(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous shard [lo, hi) of n users for `rank` (sizes differ by at most 1)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def _all_gather_vector(local: torch.Tensor, n: int, world: int) -> torch.Tensor:
    """Concatenate every rank's contiguous shard into the full vector of length n."""
    size = (n + world - 1) // world + 1
    padded = torch.zeros(size, dtype=local.dtype, device=local.device)
    padded[: local.numel()] = local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded)
    out = torch.empty(n, dtype=local.dtype, device=local.device)
    for r in range(world):
        lo, hi = shard_range(n, world, r)
        out[lo:hi] = parts[r][: hi - lo]
    return out


def _log_sum_exp2(x: np.ndarray) -> float:
    """log sum exp(2 x) with the maximum factored out."""
    a = 2.0 * np.asarray(x, np.float64)
    top = float(np.max(a))
    return top + math.log(float(np.sum(np.exp(a - top))))


def translation_tau(log_p, log_o, mass_p_sum: float, mass_o_sum: float) -> float:
    """tau of the translation step between a side P, moved by +tau, and a side O,
    moved by -tau: along that line the concave dual whose stationarity
    conditions are Eq. IPFP is const + tau dm - 1/2 e^{2 tau} P - 1/2 e^{-2 tau} O
    (P, O the sums of the sides' squared potentials, dm = sum mass_P - sum
    mass_O), maximised at tau = 1/2 log z, z the positive root of
    P z^2 - dm z - O = 0, taken in logarithms without cancellation. Non-finite
    inputs give 0."""
    lp, lo = _log_sum_exp2(log_p), _log_sum_exp2(log_o)
    dm = float(mass_p_sum - mass_o_sum)
    ln2 = math.log(2.0)
    if dm == 0.0:
        log_z = 0.5 * (lo - lp)
    else:
        big = math.log(abs(dm))
        w = 2.0 * ln2 + lp + lo - 2.0 * big
        q = 0.5 * w if w > 60.0 else (ln2 if w < -60.0 else math.log1p(math.sqrt(1.0 + math.exp(w))))
        log_z = big + q - ln2 - lp if dm > 0.0 else ln2 + lo - big - q
    tau = 0.5 * log_z
    return tau if math.isfinite(tau) else 0.0


# half_x(lo, hi, log_u_full, log_v_full) -> (new log u of X users [lo, hi), residual max of
# those rows at the entering state); half_y likewise for Y users (its residual is unused).
HalfSweep = Callable[[int, int, torch.Tensor, torch.Tensor], Tuple[torch.Tensor, float]]


def sharded_sweeps(half_x: HalfSweep, half_y: HalfSweep, log_u: torch.Tensor, log_v: torch.Tensor, sweeps: int,
                   translate: bool = False, n_sum: Optional[float] = None, m_sum: Optional[float] = None):
    """Run `sweeps` sweeps of Eq. iteration with X and Y sharded over the ranks
    (FP64 host vectors). With translate (n_sum, m_sum: the sides' capacity
    sums), the translation step precedes each half-sweep: before the u step
    log v + tau, log u - tau; before the v step log u + tau', log v - tau'.
    Returns (log_u, log_v, residual of the state entering the last sweep)."""
    world, rank = dist.get_world_size(), dist.get_rank()
    n, m = log_u.numel(), log_v.numel()
    xlo, xhi = shard_range(n, world, rank)
    ylo, yhi = shard_range(m, world, rank)
    res = torch.zeros(1, dtype=torch.float64)
    for _ in range(sweeps):
        if translate:
            tau = translation_tau(log_v.numpy(), log_u.numpy(), m_sum, n_sum)
            log_v, log_u = log_v + tau, log_u - tau
        new_u, r = half_x(xlo, xhi, log_u, log_v)
        log_u = _all_gather_vector(new_u, n, world)
        res = torch.tensor([r], dtype=torch.float64)
        dist.all_reduce(res, op=dist.ReduceOp.MAX)
        if translate:
            tau = translation_tau(log_u.numpy(), log_v.numpy(), n_sum, m_sum)
            log_u, log_v = log_u + tau, log_v - tau
        new_v, _ = half_y(ylo, yhi, log_u, log_v)
        log_v = _all_gather_vector(new_v, m, world)
    return log_u, log_v, float(res.item())


def library_half_sweeps(handle) -> Tuple[HalfSweep, HalfSweep]:
    """The two per-shard callables of :func:`sharded_sweeps` for one GPU's copy
    of the market (created with every factor and capacity, the fused path):
    each writes the gathered potentials into the market
    (tu_set_potentials_f64), runs the half-sweep of its shard
    (tu_ipfp_half_sweep_range; the u step also returns the shard's residual of
    the entering state) and reads the shard's new potentials back."""
    from . import tu_get_potentials_range_f64, tu_ipfp_half_sweep_range, tu_set_potentials_f64

    def make(side):
        def half(lo, hi, log_u, log_v):
            tu_set_potentials_f64(handle, np.ascontiguousarray(log_u.numpy()), np.ascontiguousarray(log_v.numpy()))
            res = tu_ipfp_half_sweep_range(handle, side, lo, hi, residual=side == 0)
            out = np.empty(hi - lo, np.float64)
            tu_get_potentials_range_f64(handle, side, lo, hi, out)
            return torch.from_numpy(out), (res[0] if res else 0.0)
        return half

    return make(0), make(1)
