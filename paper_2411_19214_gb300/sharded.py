"""Host schedule of one market's IPFP sweep sharded across ranks.

Within a half-sweep every user's update depends only on the other side's
fixed potentials (Eq. iteration), so the X users can be split into contiguous
shards, one per rank, each rank updating its shard against all of Y; the new
log u are then all-gathered before the Y half-sweep, which is split the same
way. The residual of the entering state (row equations of Eq. IPFP) is reduced
with a MAX all-reduce. Factors are replicated on every rank (0.5 GB at
1e6 x 1e6, d = 64). This module holds only the schedule; the per-shard
half-sweep is passed in as a callable.
"""

from __future__ import annotations

from typing import Callable, Tuple

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


HalfSweep = Callable[[int, int, torch.Tensor], Tuple[torch.Tensor, float]]


def sharded_sweeps(half_x: HalfSweep, half_y: HalfSweep, log_u: torch.Tensor, log_v: torch.Tensor, sweeps: int):
    """Run `sweeps` sweeps of Eq. iteration with X and Y sharded over the ranks.

    half_x(lo, hi, log_v_full) -> (new log u of X users [lo, hi), residual max of
    those rows for the entering state); half_y likewise for Y users against
    log u. Returns (log_u, log_v, residual of the state entering the last sweep).
    """
    world, rank = dist.get_world_size(), dist.get_rank()
    n, m = log_u.numel(), log_v.numel()
    xlo, xhi = shard_range(n, world, rank)
    ylo, yhi = shard_range(m, world, rank)
    res = torch.zeros(1, dtype=torch.float64)
    for _ in range(sweeps):
        new_u, r = half_x(xlo, xhi, log_v)
        log_u = _all_gather_vector(new_u, n, world)
        res = torch.tensor([r], dtype=torch.float64)
        dist.all_reduce(res, op=dist.ReduceOp.MAX)
        new_v, _ = half_y(ylo, yhi, log_u)
        log_v = _all_gather_vector(new_v, m, world)
    return log_u, log_v, float(res.item())
