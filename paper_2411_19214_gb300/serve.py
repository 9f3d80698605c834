"""Continuous-batching serving loop for IPFP solve requests.

One host thread drives many markets through the C ABI, each on its own CUDA
stream, so that requests arriving while others are on the GPU are admitted as
soon as memory allows and their sweeps overlap on the device:

* admission: FIFO, by the device footprint of the market
  (``tu_market_footprint``) against an HBM budget; idle resident markets are
  evicted least-recently-used first when room is needed;
* progress: every active market has at most one block of sweeps in flight
  (``tu_ipfp_sweep`` enqueues, ``tu_market_query`` checks without waiting);
  a market whose last block reports residual <= tol (row equations of
  Eq. IPFP, FP64) or that reached the sweep cap is finished;
* reply: the ranked top-k partners of every X user (``tu_topk_partners``);
* re-solves: a request that names the key of a resident market replaces its
  factors (``tu_market_update_factors``) and continues from its potentials
  (warm start) instead of starting from u = v = 1.

Latency is measured from a request's arrival time to its reply.
"""

from __future__ import annotations

import collections
import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np

from . import (tu_get_potentials, tu_ipfp_sweep, tu_market_create, tu_market_destroy, tu_market_footprint,
               tu_market_query, tu_market_update_factors, tu_topk_partners)


@dataclasses.dataclass
class SolveRequest:
    rid: int
    arrival: float            # seconds after the start of the stream
    F: object                 # N x d (torch bf16/fp32 tensor, host or device, or numpy)
    K: object
    G: object                 # M x d
    L: object
    n: np.ndarray             # N capacities (host float64)
    m: np.ndarray             # M capacities
    sigma: float
    bias_x: object = None
    bias_y: object = None
    key: Optional[str] = None  # resident-market key: a later request with the same key warm-starts

    @property
    def shape(self):
        return int(self.F.shape[0]), int(self.G.shape[0]), int(self.F.shape[1])


@dataclasses.dataclass
class SolveResult:
    rid: int
    arrival: float
    admitted: float
    finished: float
    sweeps: int
    residual: float
    converged: bool
    match_count: float
    warm: bool
    topk_idx: Optional[np.ndarray] = None
    topk_logmu: Optional[np.ndarray] = None
    log_u: Optional[np.ndarray] = None
    log_v: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclasses.dataclass
class _Slot:
    handle: int
    stream: object
    shape: tuple
    bytes: int
    req: Optional[SolveRequest] = None
    admitted: float = 0.0
    sweeps: int = 0
    start_sweeps: int = 0
    inflight: bool = False
    warm: bool = False


class Server:
    def __init__(self, hbm_budget_bytes: int, tol: float = 1e-6, max_sweeps: int = 200, sweeps_per_step: int = 8,
                 k: int = 10, max_active: int = 64, keep_potentials: bool = False):
        self.budget = int(hbm_budget_bytes)
        self.tol = tol
        self.max_sweeps = max_sweeps
        self.step = sweeps_per_step
        self.k = k
        self.max_active = max_active
        self.keep_potentials = keep_potentials
        self.used = 0
        self.resident: "collections.OrderedDict[str, _Slot]" = collections.OrderedDict()
        self.stats = dict(admitted=0, evicted=0, warm=0, not_converged=0, peak_active=0, peak_bytes=0)

    # ------------------------------------------------------------------ helpers
    def _evict_one(self) -> bool:
        if not self.resident:
            return False
        _, slot = self.resident.popitem(last=False)
        tu_market_destroy(slot.handle)
        self.used -= slot.bytes
        self.stats["evicted"] += 1
        return True

    def _admit(self, req: SolveRequest, now: float) -> Optional[_Slot]:
        import torch
        N, M, d = req.shape
        if req.key is not None and req.key in self.resident:
            slot = self.resident.pop(req.key)
            if slot.shape == (N, M, d):
                tu_market_update_factors(slot.handle, req.F, req.K, req.G, req.L)
                slot.req, slot.admitted, slot.inflight, slot.warm = req, now, False, True
                slot.start_sweeps = slot.sweeps
                self.stats["warm"] += 1
                return slot
            tu_market_destroy(slot.handle)  # shape changed: a cold solve
            self.used -= slot.bytes
        need = tu_market_footprint(N, M, d, "fused")
        while self.used + need > self.budget and self._evict_one():
            pass
        if self.used + need > self.budget:
            return None
        stream = torch.cuda.Stream()
        h = tu_market_create(req.F, req.K, req.G, req.L, req.n, req.m, req.sigma, bias_x=req.bias_x,
                             bias_y=req.bias_y, path="fused", stream=stream)
        self.used += need
        self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self.used)
        return _Slot(handle=h, stream=stream, shape=(N, M, d), bytes=need, req=req, admitted=now)

    def _finish(self, slot: _Slot, residual: float, match: float, now_fn) -> SolveResult:
        import torch
        req = slot.req
        N, M, _ = req.shape
        idx = torch.empty((N, self.k), dtype=torch.int32).pin_memory()
        lm = torch.empty((N, self.k), dtype=torch.float32).pin_memory()
        tu_topk_partners(slot.handle, 0, self.k, 0, N, idx, lm)
        lu = lv = None
        if self.keep_potentials:
            lu = np.empty(N, np.float32)
            lv = np.empty(M, np.float32)
            tu_get_potentials(slot.handle, lu, lv)
        sweeps = slot.sweeps - slot.start_sweeps
        converged = residual <= self.tol
        if not converged:
            self.stats["not_converged"] += 1
        return SolveResult(rid=req.rid, arrival=req.arrival, admitted=slot.admitted, finished=now_fn(),
                           sweeps=sweeps, residual=residual, converged=converged, match_count=match,
                           warm=slot.warm, topk_idx=idx.numpy().copy(), topk_logmu=lm.numpy().copy(),
                           log_u=lu, log_v=lv)

    # ------------------------------------------------------------------ loop
    def run(self, requests: List[SolveRequest], realtime: bool = True) -> List[SolveResult]:
        """Serve `requests` (sorted by arrival). With realtime, arrivals are
        replayed against the wall clock; otherwise all are available at once."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        now_fn = (lambda: time.perf_counter() - t0)
        nxt = 0
        pending: "collections.deque[SolveRequest]" = collections.deque()
        active: List[_Slot] = []
        results: Dict[int, SolveResult] = {}
        while len(results) < len(reqs):
            now = now_fn()
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                pending.append(reqs[nxt])
                nxt += 1
            # admission, first come first served
            while pending and len(active) < self.max_active:
                slot = self._admit(pending[0], now)
                if slot is None:
                    break
                pending.popleft()
                active.append(slot)
                self.stats["admitted"] += 1
            self.stats["peak_active"] = max(self.stats["peak_active"], len(active))
            progressed = False
            for slot in list(active):
                idle, res, match, _ = tu_market_query(slot.handle)
                if not idle:
                    continue
                if slot.inflight:
                    slot.inflight = False
                    done = slot.sweeps - slot.start_sweeps
                    if res <= self.tol or done >= self.max_sweeps:
                        key = slot.req.key
                        results[slot.req.rid] = self._finish(slot, res, match, now_fn)
                        active.remove(slot)
                        progressed = True
                        if key is not None:
                            # keep the market resident for warm-started re-solves
                            slot.req = None
                            self.resident[key] = slot
                            self.resident.move_to_end(key)
                        else:
                            tu_market_destroy(slot.handle)
                            self.used -= slot.bytes
                        continue
                n = min(self.step, self.max_sweeps - (slot.sweeps - slot.start_sweeps))
                tu_ipfp_sweep(slot.handle, n)
                slot.sweeps += n
                slot.inflight = True
                progressed = True
            if not progressed:
                time.sleep(0.0002)
        for slot in active:
            tu_market_destroy(slot.handle)
        return [results[r.rid] for r in reqs]

    def close(self):
        while self._evict_one():
            pass


def percentiles(latencies: List[float]) -> dict:
    a = np.sort(np.asarray(latencies, dtype=np.float64))
    if a.size == 0:
        return {"p50": None, "p99": None, "mean": None}
    return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "mean": float(a.mean()),
            "max": float(a[-1])}
