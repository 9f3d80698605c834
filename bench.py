#!/usr/bin/env python
"""Throughput benchmark of the IPFP sweep (one JSON line on rank 0).

Default workload: the fused mini-batch IPFP (Alg. 2) on a 1e6 x 1e6 market,
d = 64, bf16 factors N(0, 1/d), LogNormal(0, 1) popularity biases on both
sides, unit capacities, sigma = 0.5, partitions of 65536 users. One step is
one full sweep of Eq. iteration: both half-sweeps (partner preparation,
tcgen05 half-sweep, FP64 partial reduction), with the residual of the entering
state folded into the X half-sweep.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fused|dense|paper|batched|ranking|serving|dims]

N > 1 (under torchrun): every rank solves its own market of the same shape
(independent markets, weak scaling, no collective on the data path).
--impl reference times the float64 CPU oracle on the host cores on a bounded
sample of the same workload (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IPFP sweeps/s and Gpair-evals/s at 1M×1M d=64 vs plain FP32; p50/p99 solve latency"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def make_workload(name: str, rank: int, shape=None, fp8=None, sigma=None):
    from synth import dense_job_market, fused_market
    kw = {} if shape is None else {"N": shape[0], "M": shape[1]}
    if shape is not None and len(shape) > 2 and name == "fused":
        kw["d"] = shape[2]  # (profiling cases of other row lengths)
    if sigma is not None and name == "fused":
        kw["sigma"] = sigma  # (profiling cases of other exponent ranges, e.g. wide markets)
    if name == "fused" and fp8:
        # the same market with unrounded FP32 factors, quantized to e4m3 by the library
        mk = fused_market(seed=1002 + 97 * rank, dtype="fp32", **kw)
        scales = "one power-of-two scale per row" if fp8 == "rows" else "one power-of-two scale per side"
        cfg = {"workload": f"fused mini-batch IPFP (Alg. 2) with FP8 e4m3 factors ({scales}, tcgen05 "
                           "kind::f8f6f4): N=M=1,000,000 users, d=64 per factor, factors N(0,1/d), "
                           "lognormal(0,1) popularity bias on both sides, n=m=1, sigma=0.5",
               "N": mk.N, "M": mk.M, "d": mk.d, "sigma": mk.sigma, "partition": 65536, "path": "fused",
               "factors": f"e4m3, {scales}",
               "l2": "inputs larger than L2: each half-sweep streams the 128 MB partner factor matrix "
                     "(L2 is 129 MB); no flush between steps"}
        if shape is not None or sigma is not None:
            cfg["workload"] = f"fused FP8 IPFP, N={mk.N}, M={mk.M}, d={mk.d}, sigma={mk.sigma}, otherwise the same recipe"
        return mk, cfg, 65536
    if name == "fused":
        mk = fused_market(seed=1002 + 97 * rank, **kw)
        cfg = {"workload": "fused mini-batch IPFP (Alg. 2): N=M=1,000,000 users, d=64 per factor (MMA K=128), "
                           "bf16 factors N(0,1/d), lognormal(0,1) popularity bias on both sides, n=m=1, "
                           "sigma=0.5, partitions of 65,536",
               "N": mk.N, "M": mk.M, "d": mk.d, "sigma": mk.sigma, "partition": 65536, "path": "fused",
               "l2": "inputs larger than L2: each half-sweep streams the 256 MB partner factor matrix "
                     "(L2 is 129 MB); no flush between steps"}
        if shape is not None or sigma is not None:
            cfg["workload"] = (f"fused mini-batch IPFP (Alg. 2), N={mk.N}, M={mk.M}, d={mk.d}, sigma={mk.sigma}, "
                               "otherwise the same recipe")
        return mk, cfg, 65536
    if name == "dense":
        mk = dense_job_market(seed=1001 + 97 * rank, **kw)
        cfg = {"workload": "dense batch IPFP (Alg. 1) over a materialised FP32 kernel: N=20,000 candidates x "
                           "M=10,000 jobs, d=32, factors N(0,1/d), lognormal(0,1) job popularity bias, n=1, "
                           "m~U{1..5}, sigma=0.5",
               "N": mk.N, "M": mk.M, "d": mk.d, "sigma": mk.sigma, "path": "dense",
               "l2": "inputs larger than L2: each half-sweep streams the 800 MB kernel matrix "
                     "(L2 is 129 MB); no flush between steps"}
        if shape is not None:
            cfg["workload"] = f"dense batch IPFP (Alg. 1), reduced shape N={mk.N}, M={mk.M}, same recipe"
        return mk, cfg, 0
    raise ValueError(name)


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return dict(FALLBACK_PEAKS)


KERNEL_SOURCES = {
    "fused": ["paper_2411_19214_gb300/csrc/fused.cu", "paper_2411_19214_gb300/csrc/tu_internal.cuh"],
    "dense": ["paper_2411_19214_gb300/csrc/dense.cu", "paper_2411_19214_gb300/csrc/tu_internal.cuh"],
}


def source_hash(kind: str) -> str:
    """sha256 over the source files of a kernel family (ties a traffic capture to the code it measured)."""
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(entry: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
    a kernel from profiles/traffic.json, or None when there is no capture or
    the kernel's sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    e = table.get(entry)
    if not e or e.get("sha256") != source_hash(e["sources"]):
        return None
    return float(e["bytes_per_launch"])


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_index), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_median": statistics.median(power), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle on the host cores (bounded sample)
# ---------------------------------------------------------------------------

def _oracle_worker(args):
    path, rows, sigma = args
    import numpy as np

    import oracle
    F = np.load(os.path.join(path, "F.npy"), mmap_mode="r")
    K = np.load(os.path.join(path, "K.npy"), mmap_mode="r")
    G = np.load(os.path.join(path, "G.npy"), mmap_mode="r")
    L = np.load(os.path.join(path, "L.npy"), mmap_mode="r")
    bx = np.load(os.path.join(path, "bx.npy"))
    by = np.load(os.path.join(path, "by.npy"))
    n = np.load(os.path.join(path, "n.npy"))
    lv = np.zeros(G.shape[0])
    t0 = time.perf_counter()
    oracle.sampled_row_update(F, K, G, L, sigma, n, lv, rows, bx, by)
    return time.perf_counter() - t0


class OraclePool:
    """The float64 oracle's X half-sweep over sampled rows, on every host core
    (one single-threaded process per core, spawned), against all partners.
    Takes one market or a list (run() then names the market)."""

    def __init__(self, mks):
        import numpy as np
        mks = list(mks) if isinstance(mks, (list, tuple)) else [mks]
        self.dir = tempfile.mkdtemp(prefix="oracle_")
        self.dirs, self.shapes = [], []
        for i, mk in enumerate(mks):
            sub = os.path.join(self.dir, str(i))
            os.makedirs(sub)
            for name, a in (("F", mk.F), ("K", mk.K), ("G", mk.G), ("L", mk.L), ("n", mk.n), ("m", mk.m)):
                np.save(os.path.join(sub, f"{name}.npy"), a)
            np.save(os.path.join(sub, "bx.npy"), mk.bias_x if mk.bias_x is not None else np.zeros(mk.N, np.float32))
            np.save(os.path.join(sub, "by.npy"), mk.bias_y if mk.bias_y is not None else np.zeros(mk.M, np.float32))
            self.dirs.append(sub)
            self.shapes.append((mk.N, mk.M, mk.sigma))
        self.N, self.M, self.sigma = self.shapes[0]
        self.cores = os.cpu_count() or 1
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.rng = np.random.default_rng(12345)

    def run(self, rows_per_core: int, market: int = 0) -> float:
        """Wall seconds for cores x rows_per_core sampled rows of one market
        (rows_per_core at most that market's N; cores sample independently)."""
        import numpy as np
        N, _, sigma = self.shapes[market]
        tasks = []
        for _ in range(self.cores):
            rows = np.sort(self.rng.choice(N, min(rows_per_core, N), replace=False))
            tasks.append((self.dirs[market], rows, sigma))
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker, tasks)
        return time.perf_counter() - t0

    def calibrate(self, budget_s: float, market: int = 0) -> int:
        """rows per core so that one run takes about budget_s."""
        self.run(2, market)  # warm the workers (imports, page cache)
        t = self.run(4, market)
        per_row = max(t / 4.0, 1e-4)
        return max(4, int(budget_s / per_row))

    def close(self):
        import shutil
        self.pool.close()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)


def cpu_baseline(mk, budget_s: float = 15.0) -> dict:
    pool = OraclePool(mk)
    try:
        rpc = pool.calibrate(budget_s)
        t = pool.run(rpc)
        rows = rpc * pool.cores
        pairs = rows * mk.M
        pair_rate = pairs / t
        sweeps = pair_rate / (2.0 * mk.N * mk.M)
        return {"value": sweeps, "unit": "sweeps/s", "cores": pool.cores, "kind": "oracle",
                "gpair_evals_per_s": pair_rate / 1e9, "seconds": t,
                "sample": f"float64 oracle X half-sweep (Eq. iteration_minibatch) of {rows} sampled users "
                          f"against all {mk.M} partners ({pairs:.3g} pair evaluations, one process per core), "
                          f"extrapolated to 2*N*M pair evaluations per sweep"}
    finally:
        pool.close()


def run_reference(args):
    """--impl reference: the oracle as it stands, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    mk, cfg, _ = make_workload(args.workload, 0, args.shape, sigma=args.sigma)
    pool = OraclePool(mk)
    try:
        rpc = pool.calibrate(8.0)
        for _ in range(args.warmup):
            pool.run(max(1, rpc // 4))
        times = [pool.run(rpc) for _ in range(args.steps)]
    finally:
        pool.close()
    rows = rpc * pool.cores
    per_step_pairs = rows * mk.M
    total_t = sum(times)
    pair_rate = per_step_pairs * args.steps / total_t
    value = pair_rate / (2.0 * mk.N * mk.M)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "gpair_evals_per_s": pair_rate / 1e9,
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": pool.cores, "kind": "oracle",
                             "sample": f"each step: float64 oracle X half-sweep of {rows} sampled users against "
                                       f"all {mk.M} partners, one process per host core; sweeps/s extrapolated "
                                       f"to 2*N*M pair evaluations per sweep"},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def to_device_factors(mk, device, pinned=False):
    import numpy as np
    import torch

    def conv(a):
        if mk.dtype == "bf16":
            bits = (np.ascontiguousarray(a, np.float32).view(np.uint32) >> 16).astype(np.uint16)
            t = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16)
        else:
            t = torch.from_numpy(np.ascontiguousarray(a, np.float32))
        if pinned:
            return t.pin_memory()
        return t.to(device)
    return [conv(a) for a in (mk.F, mk.K, mk.G, mk.L)]


def plain_fp32_sweep(mk, dev, stream, rows_per_part: int = 8192, parts: int = 2) -> dict:
    """The comparison the method is measured against: Alg. 2 done literally in
    FP32 on the same GPU (cuBLAS SGEMM with TF32 disabled for F_j G^T + K_j L^T,
    the B x M block materialised in HBM, logsumexp, the closed-form update),
    timed on `parts` partitions of `rows_per_part` users after one warm-up
    partition and extrapolated to a full sweep (both half-sweeps cost the same
    for N = M)."""
    import math as _m

    import numpy as np
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        with torch.cuda.stream(stream):
            f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)  # noqa: E731
            F, K, G, L = f32(mk.F), f32(mk.K), f32(mk.G), f32(mk.L)
            bx = f32(mk.bias_x) if mk.bias_x is not None else torch.zeros(mk.N, device=dev)
            by = f32(mk.bias_y) if mk.bias_y is not None else torch.zeros(mk.M, device=dev)
            n = torch.from_numpy(mk.n.astype(np.float32)).to(dev)
            lv = torch.zeros(mk.M, device=dev)
            inv2s = 1.0 / (2.0 * mk.sigma)

            def partition(j0):
                j1 = min(mk.N, j0 + rows_per_part)
                logits = F[j0:j1] @ G.T
                logits.addmm_(K[j0:j1], L.T)
                logits += bx[j0:j1, None]
                logits += by[None, :]
                logits *= inv2s
                logits += lv[None, :]
                log_s = torch.logsumexp(logits, dim=1) + _m.log(0.5)
                del logits
                hl = 0.5 * torch.log(n[j0:j1])
                z = log_s - hl
                a = torch.where(z > 0, z + torch.log1p(torch.sqrt(1 + torch.exp(-2 * z))), torch.asinh(torch.exp(z)))
                return hl - a

            partition(0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for p in range(parts):
                partition((p + 1) * rows_per_part)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            del F, K, G, L
        per_row_ms = ms / (parts * rows_per_part)
        sweep_ms = per_row_ms * (mk.N + mk.M)
        return {"ms_per_sweep": sweep_ms, "sweeps_per_s": 1e3 / sweep_ms,
                "sample": f"{parts} partitions of {rows_per_part} users of the X half-sweep (Alg. 2 in FP32, cuBLAS "
                          f"SGEMM without TF32, logits materialised, logsumexp) timed with CUDA events, "
                          f"extrapolated to N + M users per sweep"}
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
        torch.cuda.empty_cache()


# offered request rates of the serving sweep and requests per rate (windows of
# about 5 s up to 50 requests/s, then 3 and 2 s)
SERVING_RATES = (20.0, 30.0, 40.0, 50.0, 100.0, 200.0)
SERVING_COUNTS = (100, 150, 200, 250, 300, 400)
WINDOW_RATES = (50.0, 100.0, 200.0)
WINDOW_COUNTS = (250, 300, 400)


def serving_block(rates, count_per_rate, budget_gb: float = 64.0, micro_batched: bool = False) -> dict:
    """Serving: Poisson streams of solve requests (sizes log-uniform in
    [1000, 200000] per side, d in {32, 64}, bf16, 30 % warm-started re-solves of
    perturbed factors) replayed in real time through the continuous-batching
    server (a stream per market), or with micro_batched through the micro-batching
    server (the requests of a 10 ms window solved together by the batched
    launch); latency from arrival to the top-10 reply. Every rate replays the
    same requests (the first `count` of one stream), arrivals scaled to the
    rate."""
    import numpy as np

    from paper_2411_19214_gb300 import serve
    from synth import serving_workload
    out = {}
    stream = serving_workload(max(count_per_rate), rate=1.0, seed=1004)

    def server():
        if micro_batched:
            return serve.WindowServer(hbm_budget_bytes=int(budget_gb * (1 << 30)), tol=1e-6, max_sweeps=200, k=10,
                                      window_s=0.01, max_batch=64)
        return serve.Server(hbm_budget_bytes=int(budget_gb * (1 << 30)), tol=1e-6, max_sweeps=200,
                            sweeps_per_step=8, k=10)

    # warm-up, untimed: the stream's first 16 requests (both row lengths, the
    # top-10 replies, the batched launch of the micro-batching server) served
    # once, so that module loading, the per-device kernel attributes and the
    # first allocations of each kind land outside the measured rates
    srv = server()
    srv.run([serve.SolveRequest(rid=w["rid"], arrival=0.0, F=w["F"], K=w["K"], G=w["G"], L=w["L"], n=w["n"],
                                m=w["m"], sigma=w["sigma"], key=None) for w in stream[:16]], realtime=False)
    srv.close()
    for rate, count in zip(rates, count_per_rate):
        reqs = [serve.SolveRequest(rid=w["rid"], arrival=w["t"] / rate, F=w["F"], K=w["K"], G=w["G"], L=w["L"],
                                   n=w["n"], m=w["m"], sigma=w["sigma"], key=w["key"]) for w in stream[:count]]
        srv = server()
        t0 = time.perf_counter()
        res = srv.run(reqs, realtime=True)
        wall = time.perf_counter() - t0
        srv.close()
        lat = serve.percentiles([r.latency for r in res])
        window = reqs[-1].arrival
        # throughput over the arrival window: replies sent before the last
        # arrival (the drain after it is one large request's service time,
        # not a rate)
        in_window = sum(r.finished <= window for r in res) / window
        # device work the loop drove: 2 N M pair evaluations per sweep plus
        # one N x M pass for the top-10 reply
        shape = {q.rid: q.shape for q in reqs}
        pair_evals = sum((2.0 * r.sweeps + 1.0) * shape[r.rid][0] * shape[r.rid][1] for r in res)
        out[f"{rate:g}/s"] = {"requests": len(res), "p50_ms": 1e3 * lat["p50"], "p99_ms": 1e3 * lat["p99"],
                              "mean_ms": 1e3 * lat["mean"], "served_in_window_per_s": in_window,
                              "served_per_s_incl_drain": len(res) / wall, "offered_per_s": rate,
                              "window_s": window, "drain_s": wall - window,
                              "not_converged_at_200_sweeps": sum(not r.converged for r in res),
                              "warm_resolves": sum(r.warm for r in res),
                              "peak_active": srv.stats.get("peak_active", srv.stats.get("largest_group")),
                              "sweeps_mean": float(np.mean([r.sweeps for r in res])),
                              "gpair_evals_per_s": pair_evals / wall / 1e9,
                              "overloaded": in_window < 0.9 * rate}
    ok = [r for r in rates if not out[f"{r:g}/s"]["overloaded"]]
    out["sustainable_per_s"] = max(ok) if ok else None  # highest offered rate served at >= 90 % in the window
    return out


def run_paper_shapes(args):
    """Sec. 4.2 of the paper: average time per IPFP iteration of the mini-batch
    method for N = M in {1e2, ..., 1e6}, D = 50, factors U[0, 1/sqrt(D)],
    n = m = 1, beta = 1 (the paper averages over I = 100 iterations). Here:
    `--steps` sweeps per size (graph replay), after `--warmup` sweeps, with
    the default launch shape and then with the shape the autotuner picks
    (tu_market_autotune: own-tile height and partner split timed on the
    market), plus two sizes between the paper's where the number of waves
    of own tiles is small and uneven (4e4: 157 tiles of 256 rows; 3e5)."""
    import torch

    import paper_2411_19214_gb300 as tu
    from synth import paper_shaped_market
    tu.load()
    tu.tu_autotune_cache_clear()
    stream = torch.cuda.Stream()

    def timed(mkt):
        mkt.sweep(args.warmup)
        mkt.sweep(args.steps)  # graph capture
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mkt.sweep(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    for N in (100, 1_000, 10_000, 40_000, 100_000, 300_000, 1_000_000):
        mk = paper_shaped_market(N)
        mkt = tu.from_synth(mk, path="fused", stream=stream)
        try:
            ms = timed(mkt)
            tune = tu.tu_market_autotune(mkt.handle, reps=3)
            ms_tuned = timed(mkt)
        finally:
            mkt.close()
        print(json.dumps({"workload": "paper-shaped mini-batch IPFP (Sec. 4.2)", "N": N, "M": N, "D": 50,
                          "ms_per_sweep": ms, "sweeps": args.steps, "gpair_evals_per_s": 2.0 * N * N / ms / 1e6,
                          "autotuned": {"ms_per_sweep": ms_tuned, "small_tiles": tune["small_tiles"],
                                        "split": tune["split"], "candidates": tune["candidates"],
                                        "gpair_evals_per_s": 2.0 * N * N / ms_tuned / 1e6},
                          "dtype": "bf16"}), flush=True)
    tu.tu_autotune_cache_clear()


BATCHED_METRIC = "aggregate Gpair-evals/s of 512 independent markets in one persistent launch per half-sweep"


def batched_config(mks) -> dict:
    return {"workload": "batched: 512 markets, N and M log-uniform in [100, 50000], d=32 bf16 N(0,1/d), "
                        "unit (even) or uniform{1..3} (odd) capacities, sigma=1",
            "markets": len(mks), "pair_evals_per_sweep": float(sum(2.0 * mk.N * mk.M for mk in mks)),
            "l2": "inputs larger than L2 (about 1 GB of packed factors); no flush"}


def run_reference_batched(args):
    """--impl reference for the batched workload: the float64 oracle's
    half-sweep over sampled users of a pair-weighted sample of the 512
    markets (the markets that carry most of the pair work), every host core,
    reported as aggregate Gpair-evals/s like the GPU line (rank 0 only)."""
    import numpy as np

    from synth import batched_markets
    if int(os.environ.get("RANK", "0")) != 0:
        return
    mks = batched_markets()
    rng = np.random.default_rng(7)
    w = np.array([float(mk.N) * mk.M for mk in mks])
    pick = rng.choice(len(mks), size=6, replace=False, p=w / w.sum())
    sub = [mks[i] for i in pick]
    pool = OraclePool(sub)
    try:
        rpc = [pool.calibrate(8.0 / len(sub), market=j) for j in range(len(sub))]
        for _ in range(args.warmup):
            pool.run(max(1, rpc[0] // 4), market=0)
        pairs, secs = 0.0, []
        for _ in range(args.steps):
            t = 0.0
            for j, mk in enumerate(sub):
                t += pool.run(rpc[j], market=j)
                pairs += pool.cores * min(rpc[j], mk.N) * mk.M
            secs.append(t)
    finally:
        pool.close()
    rate = pairs / sum(secs)
    sample = (f"each step: float64 oracle half-sweep rows of 6 markets drawn with probability proportional to "
              f"N*M ({', '.join(f'{mk.N}x{mk.M}' for mk in sub)}), sampled users against all partners, one "
              f"process per host core")
    line = {"impl": "reference", "metric": BATCHED_METRIC, "value": rate / 1e9, "unit": "Gpair-evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(secs) / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": batched_config(mks),
            "cpu_baseline": {"value": rate / 1e9, "unit": "Gpair-evals/s", "cores": pool.cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate / 1e9, "unit": "Gpair-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_paper(args):
    """--impl reference for the Sec. 4.2 shapes: the float64 oracle's time per
    sweep at N = M = 1e2 ... 1e6, from a half-sweep of sampled users on every
    host core, extrapolated to 2 N^2 pair evaluations (rank 0 only)."""
    from synth import paper_shaped_market
    if int(os.environ.get("RANK", "0")) != 0:
        return
    for N in (100, 1_000, 10_000, 100_000, 1_000_000):
        mk = paper_shaped_market(N)
        pool = OraclePool(mk)
        try:
            rpc = pool.calibrate(2.0)
            t = pool.run(rpc)
        finally:
            pool.close()
        pair_rate = pool.cores * min(rpc, N) * N / t
        ms = 2.0 * N * N / pair_rate * 1e3
        print(json.dumps({"impl": "reference", "workload": "paper-shaped mini-batch IPFP (Sec. 4.2)", "N": N, "M": N,
                          "D": 50, "ms_per_sweep": ms, "gpair_evals_per_s": pair_rate / 1e9, "dtype": "f64",
                          "cpu_baseline": {"value": ms, "unit": "ms/sweep", "cores": pool.cores, "kind": "oracle",
                                           "sample": f"float64 oracle X half-sweep of {pool.cores} x {min(rpc, N)} "
                                                     f"sampled users against all {N} partners, extrapolated"}}),
              flush=True)


def run_dims(args):
    """The paper's dimension sweep (Sec. 4.2: N = M = 1e4, time and memory
    against the factor dimension), also at 1e5 where the GPU is full: the
    Sec. 4.2 recipe (U[0, 1/sqrt(D)] factors, n = m = 1, beta = 1) for D in
    {8, 16, 32, 50, 64, 100, 128}; one JSON line per (N, D) with the time per
    sweep (`--steps` sweeps replayed as a graph after `--warmup`), the pair
    rate and the market's device footprint. The MMA inner dimension is 2D
    padded to 64, 128 or 256."""
    import torch

    import paper_2411_19214_gb300 as tu
    from synth import paper_shaped_market
    tu.load()
    stream = torch.cuda.Stream()
    for N in (10_000, 100_000):
        for D in (8, 16, 32, 50, 64, 100, 128):
            mk = paper_shaped_market(N, D=D)
            mkt = tu.from_synth(mk, path="fused", stream=stream)
            try:
                mkt.sweep(args.warmup)
                mkt.sweep(args.steps)  # graph capture
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                mkt.sweep(args.steps)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
            finally:
                mkt.close()
            kp = 64
            while kp < 2 * D:
                kp *= 2
            print(json.dumps({"workload": "dimension sweep (Sec. 4.2 recipe)", "N": N, "M": N, "D": D,
                              "mma_inner_dim": kp, "ms_per_sweep": ms, "sweeps": args.steps,
                              "gpair_evals_per_s": 2.0 * N * N / ms / 1e6,
                              "device_bytes": tu.tu_market_footprint(N, N, D, "fused"), "dtype": "bf16"}),
                  flush=True)


def run_reference_dims(args):
    """--impl reference for the dimension sweep: the float64 oracle's time per
    sweep at N = M = 1e4 for the same D, from a half-sweep of sampled users on
    every host core, extrapolated to 2 N^2 pair evaluations (rank 0 only)."""
    from synth import paper_shaped_market
    if int(os.environ.get("RANK", "0")) != 0:
        return
    N = 10_000
    for D in (8, 16, 32, 50, 64, 100, 128):
        mk = paper_shaped_market(N, D=D)
        pool = OraclePool(mk)
        try:
            rpc = pool.calibrate(2.0)
            t = pool.run(rpc)
        finally:
            pool.close()
        pair_rate = pool.cores * min(rpc, N) * N / t
        ms = 2.0 * N * N / pair_rate * 1e3
        print(json.dumps({"impl": "reference", "workload": "dimension sweep (Sec. 4.2 recipe)", "N": N, "M": N,
                          "D": D, "ms_per_sweep": ms, "gpair_evals_per_s": pair_rate / 1e9, "dtype": "f64",
                          "cpu_baseline": {"value": ms, "unit": "ms/sweep", "cores": pool.cores, "kind": "oracle",
                                           "sample": f"float64 oracle X half-sweep of {pool.cores} x {min(rpc, N)} "
                                                     f"sampled users against all {N} partners, extrapolated"}}),
              flush=True)


def run_batched(args):
    """Many independent markets in one persistent launch per half-sweep: 512
    markets, per-side sizes log-uniform in [100, 50,000], d = 32 bf16 factors
    N(0, 1/d), unit or uniform{1..3} capacities, sigma = 1. Reports (a) the
    aggregate pair-evaluation rate of K batched sweeps against the same K
    sweeps of the markets one after another (each replaying its own graph),
    (b) the solve of every market to tol 1e-6 (automatic over-relaxation,
    markets leave the launch when certified) with the tail of slow,
    near-balanced markets, (c) the roofline of the batched tensor-core kernel."""
    import numpy as np
    import torch

    import paper_2411_19214_gb300 as tu
    from synth import batched_markets
    tu.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    mks = batched_markets()
    mkts = [tu.from_synth(mk, stream=stream) for mk in mks]
    pairs = np.array([float(mk.N) * mk.M for mk in mks])
    pair_evals = 2.0 * pairs.sum()
    batch = tu.Batch(mkts, stream=stream)
    gpu_index = 0
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[0])
        except ValueError:
            pass
    try:
        for _ in range(args.warmup):
            batch.sweep(1)
        batch.sweep(args.steps)  # captures the graph the timed block replays
        torch.cuda.synchronize()
        clocks = ClockSampler(gpu_index)
        clocks.start()
        time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.sweep(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        batch.profile(True)
        batch.sweep(args.steps)
        pass_ms, passes = batch.profile_read()
        batch.profile(False)
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        seq_ms = solve_s = None
        st, infos = None, []
        if not args.no_extras:
            # the same sweeps, one market after another (each its own graph)
            for mkt in mkts:
                mkt.sweep(args.steps)
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for mkt in mkts:
                mkt.sweep(args.steps)
            s1.record(stream)
            torch.cuda.synchronize()
            seq_ms = s0.elapsed_time(s1)
            # solve every market to tol 1e-6 from u = v = 1
            for mkt in mkts:
                mkt.set_relaxation(0.0)
            batch.close()
            batch = tu.Batch(mkts, stream=stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, infos = batch.solve(tol=1e-6, max_iter=args.max_iter)
            solve_s = time.perf_counter() - t0
    finally:
        batch.close()
        for mkt in mkts:
            mkt.close()
    peaks = load_peaks()
    avg_pass_s = pass_ms / max(passes, 1) / 1e3
    flops = 2.0 * pairs.sum() * 64  # one half-sweep: 2 * N * M * (2d padded to 64) per market
    peak = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    sm_mhz = clk.get("sm_mhz") or 1900.0
    mufu_peak = 152 * 32 * sm_mhz * 1e6 / 1e12
    rate = pair_evals * args.steps / (ms / 1e3)
    traffic = measured_traffic("fused batched 512 markets d32")
    rl_tensor = {"bound": "tensor", "achieved": flops / avg_pass_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                 "frac": flops / avg_pass_s / 1e12 / peak, "traffic": traffic,
                 "kernel": "k_fused_halfsweep batched (tcgen05 BF16 MMA, K=64, + ex2 row reduction)",
                 "per_launch": f"{flops:.4g} flop in {avg_pass_s * 1e3:.3f} ms average over {passes} launches",
                 "peak_source": f"{peaks.get('source')} bf16_tflops_sustained"}
    rl_exp = {"bound": "alu", "achieved": pairs.sum() / avg_pass_s / 1e12, "peak": mufu_peak, "unit": "Tex2/s",
              "frac": pairs.sum() / avg_pass_s / 1e12 / mufu_peak, "traffic": traffic,
              "kernel": "k_fused_halfsweep batched (ex2 pipe)",
              "per_launch": f"{pairs.sum():.4g} ex2 in {avg_pass_s * 1e3:.3f} ms average over {passes} launches",
              "peak_source": "152 SMs x 32 ex2/clk/SM x sampled median SM clock"}
    # the binding unit (closest to its peak) is the roofline; the other is reported beside it
    rl_primary, rl_secondary = (rl_exp, rl_tensor) if rl_exp["frac"] > rl_tensor["frac"] else (rl_tensor, rl_exp)
    line = {"metric": BATCHED_METRIC,
            "value": rate / 1e9, "unit": "Gpair-evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic", "config": batched_config(mks),
            "roofline": rl_primary, "roofline_secondary": rl_secondary,
            "clocks": clk, "gpu_launches": 6 * args.steps + 1,
            "timing": "value: K batched sweeps replayed as one CUDA graph, CUDA events on the batch stream"}
    if seq_ms is not None:
        line["sequential"] = {"ms_per_sweep": seq_ms / args.steps,
                              "gpair_evals_per_s": pair_evals * args.steps / (seq_ms / 1e3) / 1e9,
                              "speedup_of_batched": seq_ms / ms,
                              "what": "the same sweeps, one market after another on one stream (graph per market)"}
    if infos:
        sweeps = np.array([i["sweeps"] for i in infos])
        conv = np.array([i["converged"] for i in infos])
        balance = np.array([abs(math.log(mk.N / mk.M)) for mk in mks])
        line.update({
            "solve": {"tol": 1e-6, "max_iter": args.max_iter, "relaxation": "automatic", "status": int(st),
                      "wall_s": solve_s, "converged": int(conv.sum()), "not_converged": int((~conv).sum()),
                      "sweeps_p50": float(np.percentile(sweeps, 50)), "sweeps_p90": float(np.percentile(sweeps, 90)),
                      "sweeps_p99": float(np.percentile(sweeps, 99)), "sweeps_max": int(sweeps.max()),
                      "near_balanced": int((balance < 0.1).sum()),
                      "near_balanced_sweeps_median": float(np.median(sweeps[balance < 0.1]))
                      if (balance < 0.1).any() else None,
                      "slowest": [{"N": mks[i].N, "M": mks[i].M, "sweeps": int(sweeps[i]),
                                   "converged": bool(conv[i])} for i in np.argsort(-sweeps)[:5]]}})
    return line


def run_serving(args):
    """The serving sweep of the default line on its own: one replayed stream
    of solve requests at 20 ... 200 requests/s (see serving_block)."""
    import paper_2411_19214_gb300 as tu
    tu.load()
    t0 = time.perf_counter()
    out = serving_block(SERVING_RATES, SERVING_COUNTS)
    # the alternative: micro-batches of 10 ms windows through the batched launch
    win = serving_block(WINDOW_RATES, WINDOW_COUNTS, micro_batched=True)
    print(json.dumps({"workload": "serving (continuous batching of solve requests, top-10 replies)",
                      "wall_s": time.perf_counter() - t0, "serving": out, "serving_window_batched": win,
                      "dtype": "bf16", "data": "synthetic"}),
          flush=True)


def run_ranking(args):
    """The early-stopping rule the paper proposes for practical use: sweep until
    the top-10 lists of 4,096 sampled users per side are unchanged at 3
    consecutive checks 5 sweeps apart. Reported on the fused workload's recipe
    at N = M = 100,000 (--shape to change): sweeps and wall time to the stop,
    the residual there, and how far the tight solve (tol 1e-6, automatic
    relaxation, capped) gets in the same market."""
    import torch

    import paper_2411_19214_gb300 as tu
    from synth import fused_market
    tu.load()
    N, M = args.shape if args.shape else (100_000, 100_000)
    mk = fused_market(N=N, M=M)
    stream = torch.cuda.Stream()
    mkt = tu.from_synth(mk, stream=stream)
    try:
        mkt.sweep(args.warmup)  # warm the kernels and graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = mkt.solve_ranking(k=10, sample=4096, check_every=5, patience=3, max_iter=args.max_iter)
        stop_s = time.perf_counter() - t0
        mkt.set_relaxation(0.0)
        t0 = time.perf_counter()
        tight = mkt.solve(tol=1e-6, max_iter=args.max_iter)
        tight_s = time.perf_counter() - t0
    finally:
        mkt.close()
    print(json.dumps({"workload": "ranking-stability stop (paper Sec. 4.2 discussion) on the fused recipe",
                      "N": N, "M": M, "d": mk.d, "k": 10, "sample_per_side": 4096, "check_every": 5, "patience": 3,
                      "stop": {"sweeps": info["sweeps"], "wall_s": stop_s, "residual_inf": info["residual_inf"],
                               "status": info["status"]},
                      "tight_solve_after_stop": {"tol": 1e-6, "relaxation": "automatic", "warm_start": False,
                                                 "sweeps": tight["sweeps"], "wall_s": tight_s,
                                                 "converged": tight["converged"],
                                                 "residual_inf": tight["residual_inf"]},
                      "dtype": "bf16"}), flush=True)


def solve_block(tu, h, mk, hu, hv) -> dict:
    """The workload solved to tol 1e-6 from u = v = 1 (tu_ipfp_solve, the
    translation step on, no relaxation): sweeps, wall time, the certified
    residual (row equations of Eq. IPFP, FP64 terms) and the match count from
    both sides of the returned potentials; then, for contrast, the same number
    of sweeps of Eq. iteration itself (translation step off) from u = v = 1 and
    the residual they reach."""
    import numpy as np
    t0 = time.perf_counter()
    info = tu.tu_ipfp_solve(h, 1e-6, 200, False)
    wall = time.perf_counter() - t0
    tu.tu_get_potentials(h, hu, hv)
    lu = hu.numpy().astype(np.float64)
    lv = hv.numpy().astype(np.float64)
    cx = float(np.sum(mk.n) - np.sum(np.exp(2.0 * lu)))
    cy = float(np.sum(mk.m) - np.sum(np.exp(2.0 * lv)))
    out = {"tol": 1e-6, "status": int(info["status"]), "converged": bool(info["converged"]),
           "sweeps": int(info["sweeps"]), "wall_s": wall, "residual_inf_certified": info["residual_inf"],
           "residual_l1_certified": info["residual_l1"], "match_count": info["match_count"],
           "match_count_rows": cx, "match_count_cols": cy,
           "what": "tu_ipfp_solve(tol 1e-6, warm_start 0): translation step before every half-sweep, no "
                   "relaxation; residual certified by an extra pass with FP64 terms; match counts sum n - sum u^2 "
                   "and sum m - sum v^2 of the returned potentials (FP32 copies, FP64 sums on the host)"}
    tu.tu_market_set_translation(h, False)
    tu.tu_ipfp_solve(h, 0.0, 0, False)  # u = v = 1 without sweeping
    plain = tu.tu_ipfp_sweep(h, max(1, out["sweeps"]), residual=True)
    tu.tu_market_set_translation(h, True)
    out["plain_same_sweeps_residual"] = plain
    return out


def expected_matches_block() -> dict:
    """Sec. 4.1's synthetic evaluation on the library: crowding markets of
    1,000 candidates and 500 employers (lambda in {0, 0.25, 0.5, 0.75}, d = 32,
    beta = 1), each solved to tol 1e-6 and stopped by the ranking-stability
    rule; the expected number of matches (position-based model,
    v(k) = 1 / exp(k - 1)) of both sides' top-20 lists at each stop, with the
    true like-probabilities of the generator."""
    import paper_2411_19214_gb300 as tu
    from paper_2411_19214_gb300 import evaluate
    from synth import crowding_market
    out = {}
    for lam in (0.0, 0.25, 0.5, 0.75):
        mk, P, Q = crowding_market(1000, 500, lam=lam, d=32, sigma=1.0, seed=1006)
        row = {}
        for mode in ("fixed_point", "ranking_stop"):
            mkt = tu.from_synth(mk)
            try:
                t0 = time.perf_counter()
                if mode == "fixed_point":
                    info = mkt.solve(tol=1e-6, max_iter=2000)
                else:
                    info = mkt.solve_ranking(k=20, sample=1000, check_every=1, patience=2, max_iter=2000)
                ix, _ = mkt.topk(0, 20)
                iy, _ = mkt.topk(1, 20)
                row[mode] = {"expected_matches": evaluate.expected_matches(ix.cpu().numpy(), iy.cpu().numpy(), P, Q),
                             "sweeps": int(info["sweeps"]), "residual": info["residual_inf"],
                             "wall_s": time.perf_counter() - t0}
            finally:
                mkt.close()
        out[f"lambda={lam}"] = row
    out["what"] = ("expected matches of the top-20 lists of both sides (tu_topk_partners) under the position-based "
                   "model with v(k) = 1/exp(k-1), at the fixed point (tol 1e-6) and at the ranking-stability stop "
                   "(check every sweep, patience 2); 1,000 candidates x 500 employers, crowding generator of "
                   "synth.crowding_market, beta = 1")
    return out


def quantisation_error(dev) -> dict:
    """BF16 factors against the unrounded (FP32) factors they were rounded
    from, on the fused workload's recipe at N = M = 4,000: the fused path
    solves the BF16 market and the dense FP32 path the unrounded one (both to
    1e-7 through the library); reported: relative error of mu (max and median
    over all pairs) and of the match count. Information, not a tolerance: the
    parity bars compare with the oracle on the same rounded factors."""
    import numpy as np
    import torch

    import paper_2411_19214_gb300 as tu
    from synth import fused_market
    out = {}
    mks = {"bf16": fused_market(4000, 4000, seed=1002), "fp32": fused_market(4000, 4000, seed=1002, dtype="fp32")}
    mus, counts = {}, {}
    for key, mk in mks.items():
        mkt = tu.from_synth(mk, path="fused" if key == "bf16" else "dense", device=str(dev))
        try:
            info = mkt.solve(tol=1e-7, max_iter=200)
            mus[key] = mkt.mu_block().double().cpu().numpy()
            counts[key] = info["match_count"]
            out[f"{key}_sweeps"] = info["sweeps"]
            out[f"{key}_residual"] = info["residual_inf"]
        finally:
            mkt.close()
    rel = np.abs(mus["bf16"] / mus["fp32"] - 1.0)
    out.update({"market": "fused recipe (d=64, lognormal biases both sides, sigma=0.5) at N=M=4,000",
                "mu_rel_err_max": float(rel.max()), "mu_rel_err_median": float(np.median(rel)),
                "match_count_rel_err": abs(counts["bf16"] / counts["fp32"] - 1.0),
                "what": "fused BF16 path on bf16-rounded factors vs dense FP32 path on the unrounded FP32 factors"})
    torch.cuda.synchronize()
    return out


def sub_args(args, workload: str, steps=None):
    """The arguments of a secondary workload measured inside the default run."""
    a = argparse.Namespace(**vars(args))
    a.workload = workload
    a.no_extras = False  # the secondary lines' own solve and comparison blocks are kept
    a.no_cpu_baseline = True
    a.fp8 = None
    a.partner_blocks = 0
    a.shape = None
    a.sigma = None
    if steps is not None:
        a.steps = steps
    return a


def sub_line(line) -> dict:
    """The fields of a secondary workload's line kept in the default line."""
    keep = ("metric", "value", "unit", "ms_per_step", "dtype", "config", "roofline", "roofline_secondary", "clocks",
            "e2e", "solve", "sequential", "gpu_launches", "residual_inf_after")
    return {k: line[k] for k in keep if line is not None and k in line}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2411_19214_gb300 as tu

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    tu.load()
    mk, cfg, partition = make_workload(args.workload, rank, args.shape, fp8=args.fp8, sigma=args.sigma)
    # the CPU baseline pool is spawned before the first CUDA work of this process
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mk, budget_s=args.cpu_budget)

    stream = torch.cuda.Stream()
    dev = torch.device("cuda", local)
    Fd, Kd, Gd, Ld = to_device_factors(mk, dev)
    bx = None if mk.bias_x is None else torch.from_numpy(mk.bias_x).to(dev)
    by = None if mk.bias_y is None else torch.from_numpy(mk.bias_y).to(dev)
    torch.cuda.synchronize()
    h = tu.tu_market_create(Fd, Kd, Gd, Ld, mk.n, mk.m, mk.sigma, bias_x=bx, bias_y=by,
                            path=cfg["path"], partition=partition, stream=stream, fp8=args.fp8)
    if getattr(args, "partner_blocks", 0) and cfg["path"] == "fused":
        tu.tu_market_set_partner_blocks(h, args.partner_blocks)
        cfg = dict(cfg, partner_blocks=args.partner_blocks)
    try:
        # warm-up: W single sweeps, then one untimed block of K sweeps that
        # captures the CUDA graph the timed block replays
        for _ in range(args.warmup):
            tu.tu_ipfp_sweep(h, 1)
        tu.tu_ipfp_sweep(h, args.steps)
        torch.cuda.synchronize()

        gpu_index = local
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            try:
                gpu_index = int(vis.split(",")[local])
            except ValueError:
                gpu_index = local
        clocks = ClockSampler(gpu_index)
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        time.sleep(0.3)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        tu.tu_ipfp_sweep(h, args.steps)  # K sweeps, one graph launch
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        # the same K sweeps launched directly, with a CUDA event pair around
        # every half-sweep kernel on the market's stream (roofline duration)
        tu.tu_profile_enable(h, True)
        tu.tu_ipfp_sweep(h, args.steps)
        pass_ms, passes = tu.tu_profile_read(h)
        tu.tu_profile_enable(h, False)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = ev0.elapsed_time(ev1)
        if world > 1:
            t = torch.tensor([ms], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        residual = tu.tu_ipfp_sweep(h, 0, residual=True)

        # output stage: ranked top-10 lists for every X user (one pass over N x M)
        topk_ms = None
        if not args.no_extras:
            idx = torch.empty((mk.N, 10), dtype=torch.int32, device=dev)
            lmv = torch.empty((mk.N, 10), dtype=torch.float32, device=dev)
            # warm with the full row count: it also grows the ranked lists' hand-over
            # scratch (an allocation that must stay outside the timed call)
            tu.tu_topk_partners(h, 0, 10, 0, mk.N, idx, lmv)
            torch.cuda.synchronize()
            t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0e.record(stream)
            tu.tu_topk_partners(h, 0, 10, 0, mk.N, idx, lmv)
            t1e.record(stream)
            torch.cuda.synchronize()
            topk_ms = t0e.elapsed_time(t1e)
            del idx, lmv

        # end to end through the C ABI with host buffers: H2D of the step's
        # factors from pinned memory, one sweep, D2H of the potentials
        Fh, Kh, Gh, Lh = to_device_factors(mk, dev, pinned=True)
        hu = torch.empty(mk.N, dtype=torch.float32).pin_memory()
        hv = torch.empty(mk.M, dtype=torch.float32).pin_memory()
        e2e_steps = max(1, min(args.steps, 5))
        tu.tu_market_update_factors(h, Fh, Kh, Gh, Lh)
        tu.tu_ipfp_sweep(h, 1)
        tu.tu_get_potentials(h, hu, hv)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            tu.tu_market_update_factors(h, Fh, Kh, Gh, Lh)
            tu.tu_ipfp_sweep(h, 1)
            tu.tu_get_potentials(h, hu, hv)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        elem = 2 if mk.dtype == "bf16" else 4
        h2d = 2 * (mk.N + mk.M) * mk.d * elem  # F, K (N x d) and G, L (M x d)
        d2h = (mk.N + mk.M) * 4
        solve = None
        if not args.no_extras and rank == 0:
            solve = solve_block(tu, h, mk, hu, hv)
    finally:
        tu.tu_market_destroy(h)

    # the plain FP32 blocked IPFP on the same GPU (comparison only)
    plain = None
    serving = None
    if cfg["path"] == "fused" and not args.no_extras and rank == 0 and not args.fp8:
        plain = plain_fp32_sweep(mk, dev, stream)
        serving = serving_block(SERVING_RATES, SERVING_COUNTS)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    peaks = load_peaks()
    sweeps_per_s = world * args.steps / (ms / 1e3)
    pairs_per_sweep = 2.0 * mk.N * mk.M
    avg_pass_s = pass_ms / max(passes, 1) / 1e3
    if cfg["path"] == "fused":
        kp = 2 * mk.d
        flops = 2.0 * mk.N * mk.M * kp  # one half-sweep: Phi tile products over all pairs
        achieved = flops / avg_pass_s / 1e12
        peak = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        peak_source = f"{peaks.get('source')} bf16_tflops_sustained"
        if args.fp8:
            peak *= 2.0  # e4m3 dense rate = 2 x bf16 (nominal 4.5 / 2.25 PFLOP/s)
            peak_source += " x 2 (nominal fp8/bf16 ratio)"
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "traffic": (measured_traffic(f"fused fp8 {args.fp8} 1Mx1M d64" if args.fp8
                                                 else "fused 1Mx1M d64")
                                if args.shape is None and args.sigma is None else None),
                    "kernel": "k_fused_halfsweep (tcgen05 %s MMA + ex2 row reduction)" % ("e4m3" if args.fp8
                                                                                         else "BF16"),
                    "per_launch": f"{flops:.4g} flop (2*N*M*2d) in {avg_pass_s * 1e3:.2f} ms average over "
                                  f"{passes} launches",
                    "peak_source": peak_source}
        exps = mk.N * mk.M
        sm_mhz = clk.get("sm_mhz") or 1900.0
        mufu_peak = 152 * 32 * sm_mhz * 1e6 / 1e12  # T ex2/s at the sampled clock, 32 ex2/clk/SM
        roofline_exp = {"bound": "alu", "achieved": exps / avg_pass_s / 1e12, "peak": mufu_peak,
                        "unit": "Tex2/s", "frac": exps / avg_pass_s / 1e12 / mufu_peak,
                        "peak_source": "152 SMs x 32 ex2/clk/SM x sampled median SM clock"}
    else:
        ldA = (mk.M + 3) // 4 * 4
        bytes_ = mk.N * ldA * 4.0
        achieved = bytes_ / avg_pass_s / 1e9
        peak = peaks.get("hbm_gbs")
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": measured_traffic("dense rowpass 20000x10000") if args.shape is None else None,
                    "kernel": "dense row/column pass (A-hat stream)",
                    "per_launch": f"{bytes_:.4g} B (N*ldA*4) in {avg_pass_s * 1e3:.3f} ms average over "
                                  f"{passes} launches",
                    "peak_source": f"{peaks.get('source')} hbm_gbs"}
        roofline_exp = None
    line = {"metric": METRIC, "value": sweeps_per_s, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "e4m3" if args.fp8 else mk.dtype, "data": "synthetic", "config": cfg,
            "gpair_evals_per_s": sweeps_per_s * pairs_per_sweep / 1e9,
            "residual_inf_after": residual, "sweeps_run": args.warmup + args.steps,
            "roofline": roofline,
            "clocks": clk,
            # per half-sweep: partner preparation, the pass, the FP64 reduction; per block of
            # sweeps: the two kernels that write the translation steps' offsets into the potentials
            "gpu_launches": 6 * args.steps + 2,
            "timing": "value: K sweeps replayed as one CUDA graph, CUDA events on the market stream; "
                      "roofline: the same K sweeps launched directly with an event pair per half-sweep kernel",
            "e2e": {"value": world * e2e_steps / e2e_s, "unit": "sweeps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "path": "tu_market_update_factors(pinned host F,K,G,L) + tu_ipfp_sweep(1) + "
                            "tu_get_potentials(pinned host)"}}
    if roofline_exp is not None:
        # the binding unit (closest to its peak) is the roofline; the other is reported beside it
        if roofline_exp["frac"] > roofline["frac"]:
            roofline_exp["traffic"] = roofline["traffic"]
            roofline_exp["kernel"] = roofline["kernel"]
            roofline_exp["per_launch"] = f"{exps:.4g} ex2 (N*M) in {avg_pass_s * 1e3:.2f} ms average over {passes} launches"
            roofline, roofline_exp = roofline_exp, roofline
            line["roofline"] = roofline
        line["roofline_secondary"] = roofline_exp
    if plain is not None:
        plain["speedup_of_value"] = sweeps_per_s / world / plain["sweeps_per_s"]
        line["plain_fp32"] = plain
    if serving is not None:
        line["serving"] = serving
    if topk_ms is not None:
        line["topk_all_users"] = {"ms": topk_ms, "k": 10, "users": mk.N,
                                  "gpair_evals_per_s": mk.N * mk.M / (topk_ms / 1e3) / 1e9,
                                  "vs_half_sweep": topk_ms / (avg_pass_s * 1e3),
                                  "what": "tu_topk_partners(side X, k=10) for every X user over all partners "
                                          + ("(one tensor-core pass over N x M)" if cfg["path"] == "fused" else
                                             "(one SIMT pass over the resident A-hat)")
                                          + ", after one untimed call"}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if solve is not None:
        line["solve"] = solve
    if cfg["path"] == "fused" and not args.no_extras and rank == 0 and world == 1 and args.shape is None \
            and args.sigma is None \
            and not args.fp8:
        line["quantisation_error"] = quantisation_error(dev)
        line["expected_matches"] = expected_matches_block()
        line["dense"] = sub_line(run_ours(sub_args(args, "dense")))
        line["batched"] = sub_line(run_batched(sub_args(args, "batched", steps=5)))
    if world > 1:
        dist.destroy_process_group()
    return line


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["fused", "dense", "paper", "batched", "ranking", "serving", "dims"],
                    default="fused",
                    help="paper: the Sec. 4.2 shapes (N = M = 1e2..1e6, D = 50, U[0, 1/sqrt(D)], beta = 1), "
                         "time per sweep, one JSON line per size; batched: 512 independent markets in one "
                         "persistent launch per half-sweep")
    ap.add_argument("--max-iter", type=int, default=20000, help="sweep cap of the batched solve")
    ap.add_argument("--fp8", nargs="?", const="rows", choices=["rows", "side"], default=None,
                    help="fused workload with e4m3 factors (the library quantizes the FP32 factors with "
                         "per-row power-of-two scales, or with one per side)")
    ap.add_argument("--partner-blocks", type=int, default=0,
                    help="fused workload: stream the partner matrix in this many blocks, one after another "
                         "(tu_market_set_partner_blocks), instead of the default launch shape")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain-FP32 comparison and the ranked-list timing")
    ap.add_argument("--shape", default=None,
                    help="N,M[,d] override of the workload's sizes (same recipe; for small profiling cases)")
    ap.add_argument("--sigma", type=float, default=None,
                    help="sigma override of the fused workload (same recipe; e.g. 0.01 makes its exponent range "
                         "wide: the running-maximum half-sweep)")
    args = ap.parse_args()
    if args.shape:
        args.shape = tuple(int(v) for v in args.shape.split(","))
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if (args.impl == "ours" and args.workload in ("paper", "batched", "ranking", "serving", "dims")
            and int(os.environ.get("WORLD_SIZE", "1")) > 1 and int(os.environ.get("RANK", "0")) != 0):
        return  # single-GPU workloads: rank 0 runs them (on its own device) and prints the line
    if args.workload == "paper" and args.impl == "ours":
        run_paper_shapes(args)
        return
    if args.workload == "batched" and args.impl == "ours":
        print(json.dumps(run_batched(args)), flush=True)
        return
    if args.workload == "ranking" and args.impl == "ours":
        run_ranking(args)
        return
    if args.workload == "serving" and args.impl == "ours":
        run_serving(args)
        return
    if args.workload == "dims" and args.impl == "ours":
        run_dims(args)
        return
    if args.impl == "reference" and args.workload == "dims":
        run_reference_dims(args)
        return
    if args.impl == "reference" and args.workload in ("ranking", "serving"):
        # latency and stopping-rule workloads of the GPU library; the float64
        # oracle has no serving loop and no ranking stop to time (rank 0 prints)
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps({"impl": "reference", "unavailable": f"the {args.workload} workload times the GPU "
                          "library's own loop; the float64 oracle has no counterpart"}), flush=True)
        return
    if args.impl == "reference" and args.workload == "batched":
        run_reference_batched(args)
        return
    if args.impl == "reference" and args.workload == "paper":
        run_reference_paper(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        line = run_ours(args)
        if line is not None:
            print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
