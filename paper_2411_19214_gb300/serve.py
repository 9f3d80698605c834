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
  every market sweeps with the library's translation step (``translate``; off:
  Eq. iteration exactly); with ``relax`` the market's over-relaxation factor is chosen between blocks
  by the library's automatic controller (``tu_market_relax_update``); a market
  whose last block reports residual <= tol (row equations of Eq. IPFP, FP64)
  or that reached the sweep cap is finished;
* reply: the ranked top-k partners of every X user, all M of them when a
  market has fewer than k (``tu_topk_partners`` into device buffers on the
  market's stream; a worker thread waits for them and copies them back);
* re-solves: a request that names the key of a resident market replaces its
  factors (``tu_market_update_factors``) and continues from its potentials
  (warm start) instead of starting from u = v = 1;
* failures stay with their request: a malformed request (inconsistent shapes,
  d above the fused path's limit, capacities that are not finite and
  positive, sigma <= 0, or a footprint larger than the whole budget) is
  answered ``invalid`` without being admitted; a library error while creating,
  updating or sweeping a market (non-finite factors, an exponent range the
  path refuses, a device-side wait that ran out) answers that request
  ``error`` and releases its market; a request past its ``deadline`` is
  answered ``deadline`` (after its in-flight block, without a ranking); the
  other requests are served as if it had not been there;
* tracing and metrics: each request is an NVTX range from arrival to reply
  (when torch provides start/end ranges), and with ``log_path`` every reply
  appends one JSON line (times, sweeps, residual, status).

Latency is measured from a request's arrival time to its reply.
"""

from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import json
import math
import numbers
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import (TU_ERR_UNSUPPORTED, TuError, tu_batch_create, tu_batch_destroy, tu_batch_solve, tu_get_potentials,
               tu_ipfp_solve, tu_ipfp_sweep, tu_market_create, tu_market_destroy, tu_market_footprint,
               tu_market_query, tu_market_relax_update, tu_market_set_relaxation, tu_market_set_small_tiles,
               tu_market_set_translation, tu_market_update_factors, tu_market_use_graphs, tu_topk_partners)

# the fused path's factor dimension limit (2d padded to at most 256: four 128-byte k blocks)
MAX_D = 128
# the batched launch takes packed rows of up to two k blocks (d <= 64)
MAX_D_BATCHED = 64


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
    deadline: Optional[float] = None  # seconds after arrival; past it the request is answered "deadline"

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
    # "ok" (converged), "not_converged" (sweep cap), "invalid", "error" or "deadline"
    status: str = "ok"
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _shape_of(a):
    return tuple(int(v) for v in getattr(a, "shape", ()))


def validate(req: SolveRequest) -> Optional[str]:
    """Why a request cannot be served (None when it can): host-side checks of
    shapes, capacities and sigma. Factor values are checked by the library
    (non-finite entries, exponent range) when the market is created."""
    fs, ks, gs, ls = (_shape_of(getattr(req, n)) for n in ("F", "K", "G", "L"))
    if len(fs) != 2 or fs != ks or len(gs) != 2 or gs != ls:
        return "F and K must share one N x d shape, G and L one M x d shape"
    N, d = fs
    M, dy = gs
    if N < 1 or M < 1 or d < 1 or dy != d:
        return "N, M, d must be >= 1 and both sides must have the same d"
    if d > MAX_D:
        return f"d = {d} exceeds the fused path's limit of {MAX_D}"
    for name, cap, rows in (("n", req.n, N), ("m", req.m, M)):
        c = np.asarray(cap, dtype=np.float64)
        if c.shape != (rows,):
            return f"{name} must have one capacity per user ({rows})"
        if not np.all(np.isfinite(c)) or not np.all(c > 0):
            return f"capacities {name} must be finite and > 0"
    # any real scalar (Python or numpy), not a bool, array or string
    if isinstance(req.sigma, (bool, np.bool_)) or not isinstance(req.sigma, (numbers.Real, np.floating)):
        return "sigma must be finite and > 0"
    if not (math.isfinite(float(req.sigma)) and float(req.sigma) > 0):
        return "sigma must be finite and > 0"
    for name, b, rows in (("bias_x", req.bias_x, N), ("bias_y", req.bias_y, M)):
        if b is not None and _shape_of(b) != (rows,):
            return f"{name} must have one entry per user ({rows})"
    return None


def _nvtx(kind: str, arg):
    """torch's start/end NVTX ranges (they may span loop iterations), if present."""
    try:
        import torch
        fn = getattr(torch.cuda.nvtx, "range_start" if kind == "start" else "range_end", None)
        return fn(arg) if fn is not None else None
    except Exception:  # tracing is best effort
        return None


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
    last_k: int = 0        # sweeps of the last block of this request
    r_prev: float = -1.0   # residuals read after the last two blocks (-1: none yet)
    r_last: float = -1.0


def _plan_block(last_k: int, r_prev: float, r: float, tol: float, cap: int) -> int:
    """Sweeps of a request's next block: 1 first, then at most twice the last
    block, cut to what the per-sweep decay measured over the last block needs to
    reach tol, at most ``cap`` (the policy of the library's solve loops)."""
    k = 1 if last_k <= 0 else 2 * last_k
    if last_k > 0 and r_prev > 0.0 and tol < r < r_prev and tol > 0.0:
        log_q = math.log(r / r_prev) / last_k
        need = math.ceil(math.log(tol / r) / log_q)
        if 1 <= need < k:
            k = need
    return max(1, min(k, cap))


class Server:
    def __init__(self, hbm_budget_bytes: int, tol: float = 1e-6, max_sweeps: int = 200, sweeps_per_step: int = 8,
                 k: int = 10, max_active: int = 64, keep_potentials: bool = False, relax: bool = True,
                 workers: int = 4, log_path: Optional[str] = None, translate: bool = True):
        self.budget = int(hbm_budget_bytes)
        self.tol = tol
        self.max_sweeps = max_sweeps
        self.step = sweeps_per_step
        self.k = k
        self.max_active = max_active
        self.keep_potentials = keep_potentials
        self.relax = relax
        self.translate = translate
        self.used = 0
        self.resident: "collections.OrderedDict[str, _Slot]" = collections.OrderedDict()
        self.stats = dict(admitted=0, evicted=0, warm=0, not_converged=0, peak_active=0, peak_bytes=0, invalid=0,
                          errors=0, deadline=0)
        self.pool = cf.ThreadPoolExecutor(max_workers=max(1, workers))
        self.log = open(log_path, "a") if log_path else None

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
        """Budget and residency decisions. Returns (kind, slot or bytes, future
        of the uploaded arrays), None when the budget is full for now, or
        ("invalid", reason) when the request can never fit the budget."""
        N, M, d = req.shape
        if req.key is not None and req.key in self.resident:
            slot = self.resident.pop(req.key)
            if slot.shape == (N, M, d):
                self.stats["warm"] += 1
                return ("warm", slot, self.pool.submit(self._upload, req))
            tu_market_destroy(slot.handle)  # shape changed: a cold solve
            self.used -= slot.bytes
        need = tu_market_footprint(N, M, d, "fused")
        if need > self.budget:
            return ("invalid", f"footprint {need} bytes exceeds the budget of {self.budget} bytes")
        while self.used + need > self.budget and self._evict_one():
            pass
        if self.used + need > self.budget:
            return None
        self.used += need
        self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self.used)
        return ("cold", need, self.pool.submit(self._upload, req))

    def _activate(self, kind, arg, arrays: dict, req: SolveRequest, now: float) -> _Slot:
        """Create (cold) or refresh (warm) the request's market. A library error
        propagates as TuError after the market and its bytes are released."""
        import torch
        a = arrays
        if kind == "warm":
            slot = arg
            try:
                tu_market_update_factors(slot.handle, a["F"], a["K"], a["G"], a["L"])
            except TuError:
                tu_market_destroy(slot.handle)
                self.used -= slot.bytes
                raise
            slot.req, slot.admitted, slot.inflight, slot.warm = req, now, False, True
            slot.start_sweeps = slot.sweeps
            slot.last_k, slot.r_prev, slot.r_last = 0, -1.0, -1.0
            return slot
        stream = torch.cuda.Stream()
        try:
            h = tu_market_create(a["F"], a["K"], a["G"], a["L"], req.n, req.m, req.sigma, bias_x=a["bias_x"],
                                 bias_y=a["bias_y"], path="fused", stream=stream)
        except TuError:
            self.used -= arg
            raise
        try:
            # a request runs only a few blocks of sweeps: too few to amortise a graph capture
            tu_market_use_graphs(h, False)
            # many markets share the GPU: 256-row own tiles keep the per-SM throughput
            tu_market_set_small_tiles(h, False)
            if not self.translate:
                tu_market_set_translation(h, False)  # Eq. iteration exactly
            if self.relax:
                tu_market_set_relaxation(h, 0.0)
        except TuError:
            tu_market_destroy(h)
            self.used -= arg
            raise
        return _Slot(handle=h, stream=stream, shape=req.shape, bytes=arg, req=req, admitted=now)

    def _reply(self, slot: _Slot, residual: float, match: float, now_fn):
        """Enqueue the ranked lists (and potentials) into device buffers on the
        market's stream; a worker waits for them and copies them back."""
        import torch
        req = slot.req
        N, M, _ = req.shape
        k = min(self.k, M)  # a market with fewer partners than k ranks all of them
        with torch.cuda.stream(slot.stream):
            idx = torch.empty((N, k), dtype=torch.int32, device="cuda")
            lm = torch.empty((N, k), dtype=torch.float32, device="cuda")
            lu = lv = None
            tu_topk_partners(slot.handle, 0, k, 0, N, idx, lm)
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
                               warm=slot.warm, topk_idx=host[0], topk_logmu=host[1], log_u=host[2], log_v=host[3],
                               status="ok" if residual <= tol else "not_converged")
        return self.pool.submit(fetch)

    @staticmethod
    def _failed(req: SolveRequest, status: str, error: str, now: float, admitted: float = math.nan,
                sweeps: int = 0, warm: bool = False) -> SolveResult:
        return SolveResult(rid=req.rid, arrival=req.arrival, admitted=admitted, finished=now, sweeps=sweeps,
                           residual=math.nan, converged=False, match_count=math.nan, warm=warm, status=status,
                           error=error)

    def _release(self, slot: _Slot):
        """A market whose request failed or ran out of time is not kept resident."""
        tu_market_destroy(slot.handle)
        self.used -= slot.bytes

    def _record(self, res: SolveResult, results: Dict[int, SolveResult], ranges: Dict[int, object]):
        results[res.rid] = res
        if res.status == "not_converged":
            self.stats["not_converged"] += 1
        elif res.status in ("invalid", "deadline"):
            self.stats[res.status] += 1
        elif res.status == "error":
            self.stats["errors"] += 1
        rng = ranges.pop(res.rid, None)
        if rng is not None:
            _nvtx("end", rng)
        if self.log is not None:
            self.log.write(json.dumps({
                "rid": res.rid, "status": res.status, "arrival": res.arrival, "admitted": res.admitted,
                "finished": res.finished, "latency": res.latency, "sweeps": res.sweeps,
                "residual": res.residual, "match_count": res.match_count, "warm": res.warm,
                "error": res.error}) + "\n")
            self.log.flush()

    # ------------------------------------------------------------------ loop
    def run(self, requests: List[SolveRequest], realtime: bool = True) -> List[SolveResult]:
        """Serve `requests` (sorted by arrival). With realtime, arrivals are
        replayed against the wall clock; otherwise all are available at once.
        Every request gets exactly one result (see SolveResult.status)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        now_fn = (lambda: time.perf_counter() - t0)
        nxt = 0
        pending: "collections.deque[SolveRequest]" = collections.deque()
        admitting: List[tuple] = []   # (kind, slot or bytes, future of the arrays, request)
        active: List[_Slot] = []
        finishing: List[tuple] = []   # (future of the result, slot)
        results: Dict[int, SolveResult] = {}
        ranges: Dict[int, object] = {}

        def expired(req: SolveRequest, now: float) -> bool:
            return req.deadline is not None and now > req.arrival + req.deadline

        try:
            while len(results) < len(reqs):
                now = now_fn()
                while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                    req = reqs[nxt]
                    nxt += 1
                    ranges[req.rid] = _nvtx("start", f"request {req.rid}")
                    why = validate(req)
                    if why is not None:
                        self._record(self._failed(req, "invalid", why, now), results, ranges)
                    else:
                        pending.append(req)
                progressed = False
                # requests whose deadline passed while they waited
                for req in [q for q in pending if expired(q, now)]:
                    pending.remove(req)
                    self._record(self._failed(req, "deadline", "deadline passed before admission", now), results,
                                 ranges)
                    progressed = True
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
                    progressed = True
                    if adm[0] == "invalid":
                        self._record(self._failed(req, "invalid", adm[1], now_fn()), results, ranges)
                        continue
                    admitting.append(adm + (req,))
                    busy.add(req.key)
                    self.stats["admitted"] += 1
                for x in [x for x in admitting if x[2].done()]:
                    admitting.remove(x)
                    kind, arg, fut, req = x
                    progressed = True
                    try:
                        arrays = fut.result()
                        active.append(self._activate(kind, arg, arrays, req, now_fn()))
                    except TuError as e:
                        self._record(self._failed(req, "error", str(e), now_fn()), results, ranges)
                    except Exception as e:  # an upload that failed (e.g. arrays torch cannot take)
                        if kind == "warm":
                            self._release(arg)
                        else:
                            self.used -= arg
                        self._record(self._failed(req, "error", f"{type(e).__name__}: {e}", now_fn()), results,
                                     ranges)
                self.stats["peak_active"] = max(self.stats["peak_active"], len(active) + len(admitting))
                # replies that are ready
                for fut, slot in [x for x in finishing if x[0].done()]:
                    finishing.remove((fut, slot))
                    self._record(fut.result(), results, ranges)
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
                    try:
                        idle, res, match, _ = tu_market_query(slot.handle)
                        if not idle:
                            continue
                        done = slot.sweeps - slot.start_sweeps
                        if slot.inflight:
                            slot.inflight = False
                            slot.r_prev, slot.r_last = slot.r_last, res
                            if res <= self.tol or done >= self.max_sweeps:
                                # the reply is enqueued first: if that fails, the
                                # handler below still finds the slot in `active`
                                fut = self._reply(slot, res, match, now_fn)
                                active.remove(slot)
                                finishing.append((fut, slot))
                                progressed = True
                                continue
                        if expired(slot.req, now_fn()):
                            active.remove(slot)
                            self._release(slot)
                            self._record(self._failed(slot.req, "deadline", "deadline passed during the solve",
                                                      now_fn(), slot.admitted, done, slot.warm), results, ranges)
                            progressed = True
                            continue
                        if slot.inflight is False and done > 0 and self.relax:
                            tu_market_relax_update(slot.handle, self.tol)
                        n = min(_plan_block(slot.last_k, slot.r_prev, slot.r_last, self.tol, self.step),
                                self.max_sweeps - done)
                        tu_ipfp_sweep(slot.handle, n)
                        slot.sweeps += n
                        slot.last_k = n
                        slot.inflight = True
                        progressed = True
                    except TuError as e:
                        active.remove(slot)
                        self._release(slot)
                        self._record(self._failed(slot.req, "error", str(e), now_fn(), slot.admitted,
                                                  slot.sweeps - slot.start_sweeps, slot.warm), results, ranges)
                        progressed = True
                if not progressed:
                    time.sleep(0.0002)
        finally:
            for x in admitting:
                try:
                    x[2].result()
                except Exception:
                    pass
                if x[0] == "warm":
                    active.append(x[1])
                else:
                    self.used -= x[1]
            for fut, slot in finishing:
                try:
                    fut.result()
                except Exception:
                    pass
                active.append(slot)
            for slot in active:
                tu_market_destroy(slot.handle)
                self.used -= slot.bytes
            for rng in ranges.values():
                if rng is not None:
                    _nvtx("end", rng)
        return [results[r.rid] for r in reqs]

    def close(self):
        while self._evict_one():
            pass
        self.pool.shutdown(wait=True)
        if self.log is not None:
            self.log.close()
            self.log = None


def percentiles(latencies: List[float]) -> dict:
    a = np.sort(np.asarray(latencies, dtype=np.float64))
    if a.size == 0:
        return {"p50": None, "p99": None, "mean": None}
    return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "mean": float(a.mean()),
            "max": float(a[-1])}


class WindowServer:
    """Micro-batching over the batched persistent launch, the alternative to
    :class:`Server`'s stream per market: requests that arrive within
    ``window_s`` of the oldest waiting one (at most ``max_batch``) are made
    markets on one stream, grouped by packed row length (d <= 32: 64
    elements, else 128), and each group is solved by ``tu_batch_solve``: one
    persistent launch per half-sweep for the whole group, converged markets
    leaving it; then every request gets its top-k reply. A re-solve of a
    resident market (same key and shape) replaces its factors and joins its
    group from its current potentials (new markets start from u = v = 1).
    Admission by HBM footprint with LRU eviction of idle resident markets,
    and validation, as in Server. The host thread blocks in the batched
    solve, so requests that arrive meanwhile wait for the next window. d above
    the batched launch's limit (64) is answered ``invalid``; a group that the
    batched launch refuses (a market with a wide exponent range) is solved
    market by market (``tu_ipfp_solve``), so that one such request does not
    fail the others."""

    def __init__(self, hbm_budget_bytes: int, tol: float = 1e-6, max_sweeps: int = 200, k: int = 10,
                 window_s: float = 0.01, max_batch: int = 64, relax: bool = True, translate: bool = True):
        import torch
        self.budget = int(hbm_budget_bytes)
        self.tol = tol
        self.max_sweeps = max_sweeps
        self.k = k
        self.window = window_s
        self.max_batch = max_batch
        self.relax = relax
        self.translate = translate
        self.used = 0
        self.resident: "collections.OrderedDict[str, tuple]" = collections.OrderedDict()  # key -> (handle, shape, bytes)
        self.stream = torch.cuda.Stream()
        self.stats = dict(admitted=0, evicted=0, warm=0, groups=0, largest_group=0, invalid=0, errors=0,
                          solved_alone=0)

    def _evict_one(self) -> bool:
        if not self.resident:
            return False
        _, (h, _, nbytes) = self.resident.popitem(last=False)
        tu_market_destroy(h)
        self.used -= nbytes
        self.stats["evicted"] += 1
        return True

    def _market(self, req: SolveRequest):
        """(handle, bytes, warm) of the request's market, or a failure string."""
        N, M, d = req.shape
        if req.key is not None and req.key in self.resident:
            h, shape, nbytes = self.resident.pop(req.key)
            if shape == req.shape:
                try:
                    tu_market_update_factors(h, *(np.ascontiguousarray(getattr(req, a)) for a in "FKGL"))
                except TuError as e:
                    tu_market_destroy(h)
                    self.used -= nbytes
                    return f"error: {e}"
                self.stats["warm"] += 1
                return h, nbytes, True
            tu_market_destroy(h)
            self.used -= nbytes
        need = tu_market_footprint(N, M, d, "fused")
        if need > self.budget:
            return f"invalid: footprint {need} bytes exceeds the budget of {self.budget} bytes"
        while self.used + need > self.budget and self._evict_one():
            pass
        if self.used + need > self.budget:
            return "wait"
        try:
            h = tu_market_create(*(np.ascontiguousarray(getattr(req, a)) for a in "FKGL"), req.n, req.m, req.sigma,
                                 bias_x=req.bias_x, bias_y=req.bias_y, path="fused", stream=self.stream)
        except TuError as e:
            return f"error: {e}"
        try:
            if not self.translate:
                tu_market_set_translation(h, False)
            if self.relax:
                tu_market_set_relaxation(h, 0.0)
        except TuError as e:
            tu_market_destroy(h)
            return f"error: {e}"
        self.used += need
        return h, need, False

    def _solve_alone(self, made, now_fn, results) -> list:
        """The markets of a group one by one (tu_ipfp_solve); None in place of
        a market whose solve failed, which is answered and released here."""
        infos = []
        for req, h, nbytes, warm, adm in made:
            self.stats["solved_alone"] += 1
            try:
                infos.append(tu_ipfp_solve(h, self.tol, self.max_sweeps, warm_start=True))
            except TuError as e:
                tu_market_destroy(h)
                self.used -= nbytes
                self.stats["errors"] += 1
                results[req.rid] = Server._failed(req, "error", str(e), now_fn(), adm, 0, warm)
                infos.append(None)
        return infos

    def _solve_group(self, group, now_fn, results) -> list:
        """Solve one group; returns the requests that found no room yet."""
        made = []  # (req, handle, bytes, warm, admitted)
        deferred = []
        for req in group:
            now = now_fn()
            r = self._market(req)
            if r == "wait":
                deferred.append(req)
                continue
            if isinstance(r, str):
                status = "invalid" if r.startswith("invalid") else "error"
                self.stats["invalid" if status == "invalid" else "errors"] += 1
                results[req.rid] = Server._failed(req, status, r.split(": ", 1)[-1], now)
                continue
            self.stats["admitted"] += 1
            made.append((req, r[0], r[1], r[2], now))
        if not made:
            return deferred
        self.stats["groups"] += 1
        self.stats["largest_group"] = max(self.stats["largest_group"], len(made))
        try:
            try:
                b = tu_batch_create([x[1] for x in made], stream=self.stream)
                try:
                    _, infos = tu_batch_solve(b, self.tol, self.max_sweeps, len(made), warm_start=True)
                finally:
                    tu_batch_destroy(b)
            except TuError as e:
                if e.status != TU_ERR_UNSUPPORTED:
                    raise
                # a market the batched launch cannot take (a wide exponent
                # range): every market of the group is solved on its own
                infos = self._solve_alone(made, now_fn, results)
        except TuError as e:
            for req, h, nbytes, warm, adm in made:
                tu_market_destroy(h)
                self.used -= nbytes
                self.stats["errors"] += 1
                results[req.rid] = Server._failed(req, "error", str(e), now_fn(), adm, 0, warm)
            return deferred
        for (req, h, nbytes, warm, adm), info in zip(made, infos):
            if info is None:  # failed alone: already answered and released
                continue
            N, M, _ = req.shape
            k = min(self.k, M)
            idx = np.empty((N, k), np.int32)
            lm = np.empty((N, k), np.float32)
            try:
                tu_topk_partners(h, 0, k, 0, N, idx, lm)
            except TuError as e:
                tu_market_destroy(h)
                self.used -= nbytes
                results[req.rid] = Server._failed(req, "error", str(e), now_fn(), adm, info["sweeps"], warm)
                continue
            ok = info["residual_inf"] <= self.tol
            results[req.rid] = SolveResult(rid=req.rid, arrival=req.arrival, admitted=adm, finished=now_fn(),
                                           sweeps=info["sweeps"], residual=info["residual_inf"], converged=ok,
                                           match_count=info["match_count"], warm=warm, topk_idx=idx,
                                           topk_logmu=lm, status="ok" if ok else "not_converged")
            if req.key is not None:
                self.resident[req.key] = (h, req.shape, nbytes)
            else:
                tu_market_destroy(h)
                self.used -= nbytes
        return deferred

    def run(self, requests: List[SolveRequest], realtime: bool = True) -> List[SolveResult]:
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        now_fn = (lambda: time.perf_counter() - t0)
        nxt = 0
        pending: List[SolveRequest] = []
        results: Dict[int, SolveResult] = {}
        while len(results) < len(reqs):
            now = now_fn()
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                req = reqs[nxt]
                nxt += 1
                why = validate(req)
                if why is None and req.shape[2] > MAX_D_BATCHED:
                    why = f"d = {req.shape[2]} exceeds the batched launch's limit of {MAX_D_BATCHED}"
                if why is not None:
                    self.stats["invalid"] += 1
                    results[req.rid] = Server._failed(req, "invalid", why, now)
                else:
                    pending.append(req)
            full = len(pending) >= self.max_batch
            due = pending and (now - pending[0].arrival >= self.window or nxt == len(reqs) or not realtime)
            if not (full or due):
                time.sleep(0.0002)
                continue
            take, pending = pending[:self.max_batch], pending[self.max_batch:]
            # a key may appear once per group (its market is one member)
            seen, group, later = set(), [], []
            for q in take:
                if q.key is not None and q.key in seen:
                    later.append(q)
                else:
                    seen.add(q.key)
                    group.append(q)
            for narrow in (True, False):
                part = [q for q in group if (q.shape[2] <= 32) == narrow]
                if part:
                    later += self._solve_group(part, now_fn, results)
            pending = sorted(later, key=lambda r: r.arrival) + pending
        return [results[r.rid] for r in reqs]

    def close(self):
        while self._evict_one():
            pass
