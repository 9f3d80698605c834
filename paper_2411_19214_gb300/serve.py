"""Continuous-batching serving loop for IPFP solve requests.

One host thread drives many markets through the C ABI, each on its own CUDA
stream, so that requests arriving while others are on the GPU are admitted as
soon as memory allows and their sweeps overlap on the device:

* admission: FIFO, by the device footprint of the market
  (``tu_market_footprint``) against an HBM budget; idle resident markets are
  evicted least-recently-used first when room is needed. A request's factors
  come from host memory, which for large requests takes tens of milliseconds
  of host time to move, so worker threads stage them on the device (pinned
  copies with torch) while the main loop keeps the other markets' sweeps
  flowing; the market is then created from device pointers;
* progress: every active market has at most one block of sweeps in flight
  (``tu_ipfp_sweep`` enqueues, ``tu_market_query`` checks without waiting);
  with ``relax`` the market's over-relaxation factor is chosen between blocks
  by the library's automatic controller (``tu_market_relax_update``); a market
  whose last block reports residual <= tol (row equations of Eq. IPFP, FP64)
  or that reached the sweep cap is finished;
* reply: the ranked top-k partners of every X user (``tu_topk_partners``
  into device buffers on the market's stream; a worker thread waits for them
  and copies them back);
* re-solves: a request that names the key of a resident market replaces its
  factors (``tu_market_update_factors``) and continues from its potentials
  (warm start) instead of starting from u = v = 1.

Latency is measured from a request's arrival time to its reply.
"""

from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import (tu_get_potentials, tu_ipfp_sweep, tu_market_create, tu_market_destroy, tu_market_footprint,
               tu_market_query, tu_market_relax_update, tu_market_set_relaxation, tu_market_update_factors,
               tu_market_use_graphs, tu_topk_partners)


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
                 k: int = 10, max_active: int = 64, keep_potentials: bool = False, relax: bool = True,
                 workers: int = 4):
        self.budget = int(hbm_budget_bytes)
        self.tol = tol
        self.max_sweeps = max_sweeps
        self.step = sweeps_per_step
        self.k = k
        self.max_active = max_active
        self.keep_potentials = keep_potentials
        self.relax = relax
        self.used = 0
        self.resident: "collections.OrderedDict[str, _Slot]" = collections.OrderedDict()
        self.stats = dict(admitted=0, evicted=0, warm=0, not_converged=0, peak_active=0, peak_bytes=0)
        self.pool = cf.ThreadPoolExecutor(max_workers=max(1, workers))

    # ------------------------------------------------------------------ helpers
    # Every library call is made from the thread that runs run(); the workers
    # only move data between host and device with torch (uploads of request
    # factors, downloads of replies), which is where a large request spends
    # tens of milliseconds of host time.
    def _evict_one(self) -> bool:
        if not self.resident:
            return False
        _, slot = self.resident.popitem(last=False)
        tu_market_destroy(slot.handle)
        self.used -= slot.bytes
        self.stats["evicted"] += 1
        return True

    _local = threading.local()

    @classmethod
    def _upload(cls, req: SolveRequest) -> dict:
        """Worker thread: the request's arrays on the device (pinned staging, the
        worker's own side stream)."""
        import torch
        if not hasattr(cls._local, "side"):
            torch.cuda.set_device(0)
            cls._local.side = torch.cuda.Stream()
        side = cls._local.side
        out = {}
        with torch.cuda.stream(side):
            for name in ("F", "K", "G", "L", "bias_x", "bias_y"):
                a = getattr(req, name)
                if a is None:
                    out[name] = None
                    continue
                t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
                if not t.is_cuda:
                    t = t.pin_memory().to("cuda", non_blocking=True)
                out[name] = t
        side.synchronize()
        return out

    def _admit(self, req: SolveRequest):
        """Budget and residency decisions. Returns (kind, slot, future of the
        uploaded arrays), or None when the budget is full."""
        N, M, d = req.shape
        if req.key is not None and req.key in self.resident:
            slot = self.resident.pop(req.key)
            if slot.shape == (N, M, d):
                self.stats["warm"] += 1
                return ("warm", slot, self.pool.submit(self._upload, req))
            tu_market_destroy(slot.handle)  # shape changed: a cold solve
            self.used -= slot.bytes
        need = tu_market_footprint(N, M, d, "fused")
        while self.used + need > self.budget and self._evict_one():
            pass
        if self.used + need > self.budget:
            return None
        self.used += need
        self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self.used)
        return ("cold", need, self.pool.submit(self._upload, req))

    def _activate(self, kind, arg, arrays: dict, req: SolveRequest, now: float) -> _Slot:
        import torch
        a = arrays
        if kind == "warm":
            slot = arg
            tu_market_update_factors(slot.handle, a["F"], a["K"], a["G"], a["L"])
            slot.req, slot.admitted, slot.inflight, slot.warm = req, now, False, True
            slot.start_sweeps = slot.sweeps
            return slot
        stream = torch.cuda.Stream()
        h = tu_market_create(a["F"], a["K"], a["G"], a["L"], req.n, req.m, req.sigma, bias_x=a["bias_x"],
                             bias_y=a["bias_y"], path="fused", stream=stream)
        # a request runs only a few blocks of sweeps: too few to amortise a graph capture
        tu_market_use_graphs(h, False)
        if self.relax:
            tu_market_set_relaxation(h, 0.0)
        return _Slot(handle=h, stream=stream, shape=req.shape, bytes=arg, req=req, admitted=now)

    def _reply(self, slot: _Slot, residual: float, match: float, now_fn):
        """Enqueue the ranked lists (and potentials) into device buffers on the
        market's stream; a worker waits for them and copies them back."""
        import torch
        req = slot.req
        N, M, _ = req.shape
        with torch.cuda.stream(slot.stream):
            idx = torch.empty((N, self.k), dtype=torch.int32, device="cuda")
            lm = torch.empty((N, self.k), dtype=torch.float32, device="cuda")
            lu = lv = None
            tu_topk_partners(slot.handle, 0, self.k, 0, N, idx, lm)
            if self.keep_potentials:
                lu = torch.empty(N, dtype=torch.float32, device="cuda")
                lv = torch.empty(M, dtype=torch.float32, device="cuda")
                tu_get_potentials(slot.handle, lu, lv)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        sweeps = slot.sweeps - slot.start_sweeps
        tol = self.tol

        def fetch() -> SolveResult:
            ev.synchronize()
            host = [None if t is None else t.cpu().numpy() for t in (idx, lm, lu, lv)]
            return SolveResult(rid=req.rid, arrival=req.arrival, admitted=slot.admitted, finished=now_fn(),
                               sweeps=sweeps, residual=residual, converged=residual <= tol, match_count=match,
                               warm=slot.warm, topk_idx=host[0], topk_logmu=host[1], log_u=host[2], log_v=host[3])
        return self.pool.submit(fetch)

    # ------------------------------------------------------------------ loop
    def run(self, requests: List[SolveRequest], realtime: bool = True) -> List[SolveResult]:
        """Serve `requests` (sorted by arrival). With realtime, arrivals are
        replayed against the wall clock; otherwise all are available at once."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        now_fn = (lambda: time.perf_counter() - t0)
        nxt = 0
        pending: "collections.deque[SolveRequest]" = collections.deque()
        admitting: List[tuple] = []   # (kind, slot or bytes, future of the arrays, request)
        active: List[_Slot] = []
        finishing: List[tuple] = []   # (future of the result, slot)
        results: Dict[int, SolveResult] = {}
        try:
            while len(results) < len(reqs):
                now = now_fn()
                while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                    pending.append(reqs[nxt])
                    nxt += 1
                progressed = False
                # admission, first come first served; a request whose key names a
                # market that is still in use waits until it is resident again
                busy = {sl.req.key for sl in active} | {x[3].key for x in admitting} | \
                       {sl.req.key for _, sl in finishing}
                while pending and len(active) + len(admitting) < self.max_active:
                    if pending[0].key is not None and pending[0].key in busy:
                        break
                    adm = self._admit(pending[0])
                    if adm is None:
                        break
                    req = pending.popleft()
                    admitting.append(adm + (req,))
                    busy.add(req.key)
                    self.stats["admitted"] += 1
                    progressed = True
                for x in [x for x in admitting if x[2].done()]:
                    admitting.remove(x)
                    active.append(self._activate(x[0], x[1], x[2].result(), x[3], now_fn()))
                    progressed = True
                self.stats["peak_active"] = max(self.stats["peak_active"], len(active) + len(admitting))
                # replies that are ready
                for fut, slot in [x for x in finishing if x[0].done()]:
                    finishing.remove((fut, slot))
                    res = fut.result()
                    results[res.rid] = res
                    if not res.converged:
                        self.stats["not_converged"] += 1
                    key = slot.req.key
                    if key is not None:
                        # keep the market resident for warm-started re-solves
                        slot.req = None
                        self.resident[key] = slot
                        self.resident.move_to_end(key)
                    else:
                        tu_market_destroy(slot.handle)
                        self.used -= slot.bytes
                    progressed = True
                for slot in list(active):
                    idle, res, match, _ = tu_market_query(slot.handle)
                    if not idle:
                        continue
                    if slot.inflight:
                        slot.inflight = False
                        done = slot.sweeps - slot.start_sweeps
                        if res <= self.tol or done >= self.max_sweeps:
                            active.remove(slot)
                            finishing.append((self._reply(slot, res, match, now_fn), slot))
                            progressed = True
                            continue
                        if self.relax:
                            tu_market_relax_update(slot.handle, self.tol)
                    n = min(self.step, self.max_sweeps - (slot.sweeps - slot.start_sweeps))
                    tu_ipfp_sweep(slot.handle, n)
                    slot.sweeps += n
                    slot.inflight = True
                    progressed = True
                if not progressed:
                    time.sleep(0.0002)
        finally:
            for x in admitting:
                x[2].result()
                if x[0] == "warm":
                    active.append(x[1])
                else:
                    self.used -= x[1]
            for fut, slot in finishing:
                fut.result()
                active.append(slot)
            for slot in active:
                tu_market_destroy(slot.handle)
                self.used -= slot.bytes
        return [results[r.rid] for r in reqs]

    def close(self):
        while self._evict_one():
            pass
        self.pool.shutdown(wait=True)


def percentiles(latencies: List[float]) -> dict:
    a = np.sort(np.asarray(latencies, dtype=np.float64))
    if a.size == 0:
        return {"p50": None, "p99": None, "mean": None}
    return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "mean": float(a.mean()),
            "max": float(a[-1])}
