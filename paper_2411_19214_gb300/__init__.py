"""Python binding of libtu_ipfp.so (C ABI in include/tu_ipfp.h).

The binding only marshals arguments: every step of the IPFP runs in the CUDA
library. Functions carry the C names (``tu_market_create``, ``tu_ipfp_sweep``,
``tu_ipfp_solve``, ``tu_mu_block``, ``tu_topk_partners``,
``tu_get_potentials``, ``tu_set_potentials``, ``tu_market_update_factors``,
``tu_market_destroy``); :class:`Market` wraps them for convenience. Arrays may
be torch tensors (CPU or CUDA) or numpy arrays; the library detects host or
device memory itself. There is no CPU fallback: without the built library
every call raises.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np


TU_OK, TU_ERR_INVALID_ARG, TU_ERR_OOM, TU_ERR_CUDA, TU_ERR_NOT_CONVERGED, TU_ERR_NONFINITE, TU_ERR_TIMEOUT, \
    TU_ERR_UNSUPPORTED = range(8)
TU_DTYPE_BF16, TU_DTYPE_FP32, TU_DTYPE_FP8E4M3, TU_DTYPE_FP8E4M3_SIDE = 0, 1, 2, 3
TU_PATH_FUSED, TU_PATH_DENSE = 0, 1

# where build.py puts the library (kept in step with build.LIB)
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libtu_ipfp.so")
_lib = None


class MarketDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("M", ctypes.c_int64), ("d", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("path", ctypes.c_int32),
                ("F", ctypes.c_void_p), ("K", ctypes.c_void_p), ("G", ctypes.c_void_p), ("L", ctypes.c_void_p),
                ("bias_x", ctypes.c_void_p), ("bias_y", ctypes.c_void_p),
                ("n", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("sigma", ctypes.c_double), ("partition", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("fscale_x", ctypes.c_void_p), ("fscale_y", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("status", ctypes.c_int32), ("residual_inf", ctypes.c_double),
                ("residual_l1", ctypes.c_double), ("match_count", ctypes.c_double)]


class TuneInfo(ctypes.Structure):
    _fields_ = [("small_tiles", ctypes.c_int32), ("split", ctypes.c_int32), ("ms", ctypes.c_double),
                ("ms_default", ctypes.c_double), ("candidates", ctypes.c_int32)]


class TuError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = status_string(status) if _lib is not None else str(status)
        super().__init__(f"{where}: {name}" + (f" ({detail})" if detail else ""))


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load the shared library (it must have been built: see build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -m paper_2411_19214_gb300.build`")
    lib = ctypes.CDLL(p)
    V, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sigs = {
        "tu_market_create": (I32, [ctypes.POINTER(MarketDesc), ctypes.POINTER(V)]),
        "tu_market_update_factors": (I32, [V, V, V, V, V]),
        "tu_market_update_factors_fp8": (I32, [V, V, V, V, V, V, V]),
        "tu_ipfp_sweep": (I32, [V, I32, ctypes.POINTER(D)]),
        "tu_ipfp_solve": (I32, [V, D, I32, I32, ctypes.POINTER(SolveInfo)]),
        "tu_ipfp_solve_ranking": (I32, [V, I32, I64, I32, I32, D, I32, I32, ctypes.POINTER(SolveInfo)]),
        "tu_mu_block": (I32, [V, I64, I64, I64, I64, V, I64]),
        "tu_topk_partners": (I32, [V, I32, I32, I64, I64, V, V]),
        "tu_get_potentials": (I32, [V, V, V]),
        "tu_get_potentials_f64": (I32, [V, V, V]),
        "tu_get_potentials_range_f64": (I32, [V, I32, I64, I64, V]),
        "tu_ipfp_half_sweep_range": (I32, [V, I32, I64, I64, ctypes.POINTER(D)]),
        "tu_set_potentials_f64": (I32, [V, V, V]),
        "tu_set_potentials": (I32, [V, V, V]),
        "tu_fused_halfsweep_noalloc": (I32, [I64, I64, I64, V, V, V, V, V, V, V, D, V, ctypes.POINTER(D), V]),
        "tu_market_set_relaxation": (I32, [V, D]),
        "tu_market_relax_update": (I32, [V, D]),
        "tu_market_use_graphs": (I32, [V, I32]),
        "tu_selftest_wait_timeout": (I32, [D, ctypes.POINTER(D)]),
        "tu_set_checked_mode": (I32, [I32]),
        "tu_market_set_small_tiles": (I32, [V, I32]),
        "tu_market_set_split": (I32, [V, I32]),
        "tu_market_get_shape": (I32, [V, ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "tu_market_set_partner_blocks": (I32, [V, I32]),
        "tu_market_autotune": (I32, [V, I32, ctypes.POINTER(TuneInfo)]),
        "tu_autotune_cache_save": (I32, [ctypes.c_char_p]),
        "tu_autotune_cache_load": (I32, [ctypes.c_char_p]),
        "tu_autotune_cache_clear": (None, []),
        "tu_market_set_translation": (I32, [V, I32]),
        "tu_relax_schedule": (I32, [D, D, V, V, I32, V]),
        "tu_guard_violations": (I64, [ctypes.c_char_p, I64]),
        "tu_market_query": (I32, [V, ctypes.POINTER(I32), ctypes.POINTER(D), ctypes.POINTER(D),
                                  ctypes.POINTER(I64)]),
        "tu_market_footprint": (I64, [I64, I64, I64, I32]),
        "tu_profile_enable": (I32, [V, I32]),
        "tu_profile_read": (I32, [V, ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "tu_market_destroy": (None, [V]),
        "tu_status_string": (ctypes.c_char_p, [I32]),
        "tu_market_last_error": (ctypes.c_char_p, [V]),
        "tu_batch_create": (I32, [ctypes.POINTER(V), I32, V, ctypes.POINTER(V)]),
        "tu_batch_sweep": (I32, [V, I32, V]),
        "tu_batch_solve": (I32, [V, D, I32, I32, ctypes.POINTER(SolveInfo)]),
        "tu_batch_profile_enable": (I32, [V, I32]),
        "tu_batch_profile_read": (I32, [V, ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "tu_batch_destroy": (None, [V]),
        "tu_batch_last_error": (ctypes.c_char_p, [V]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list:
    """Names of the ABI functions the loaded library exports."""
    lib = load()
    names = ["tu_market_create", "tu_market_update_factors", "tu_market_update_factors_fp8", "tu_ipfp_sweep",
             "tu_ipfp_solve",
             "tu_ipfp_solve_ranking", "tu_mu_block",
             "tu_topk_partners", "tu_get_potentials", "tu_set_potentials", "tu_profile_enable",
             "tu_profile_read", "tu_market_destroy", "tu_status_string", "tu_market_last_error",
             "tu_batch_create", "tu_batch_sweep", "tu_batch_solve", "tu_batch_profile_enable",
             "tu_batch_profile_read", "tu_batch_destroy", "tu_batch_last_error"]
    return [n for n in names if hasattr(lib, n)]


def status_string(status: int) -> str:
    return load().tu_status_string(int(status)).decode()


# ---------------------------------------------------------------------------
# argument marshalling
# ---------------------------------------------------------------------------

def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensors passed to the library must be contiguous")
            return a.data_ptr()
    except ImportError:  # pragma: no cover
        pass
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return a.ctypes.data
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)!r}")


def _dtype_code(a) -> int:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype == torch.bfloat16:
                return TU_DTYPE_BF16
            if a.dtype == torch.float32:
                return TU_DTYPE_FP32
            raise TypeError(f"factor dtype {a.dtype} not supported (bfloat16 or float32)")
    except ImportError:  # pragma: no cover
        pass
    if a.dtype == np.uint16:
        return TU_DTYPE_BF16
    if a.dtype == np.float32:
        return TU_DTYPE_FP32
    raise TypeError(f"factor dtype {a.dtype} not supported (uint16 bf16 bits or float32)")


def _shape(a):
    return tuple(int(s) for s in a.shape)


def _check(status: int, where: str, handle=None, batch=False):
    if status != TU_OK:
        detail = ""
        if handle:
            lib = load()
            raw = lib.tu_batch_last_error(handle) if batch else lib.tu_market_last_error(handle)
            detail = raw.decode() if raw else ""
        raise TuError(status, where, detail)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---------------------------------------------------------------------------
# the C functions, same names
# ---------------------------------------------------------------------------

def _is_bytes(a) -> bool:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.dtype == torch.uint8
    except ImportError:  # pragma: no cover
        pass
    return isinstance(a, np.ndarray) and a.dtype == np.uint8


def tu_market_create(F, K, G, L, n, m, sigma: float, *, bias_x=None, bias_y=None, path: str = "fused",
                     partition: int = 0, stream=None, fp8: bool = False, fscale_x=None, fscale_y=None) -> int:
    """Create a market; returns the opaque handle (int). n, m: host float64.
    fp8: compute with e4m3 factors. True (or "rows"): per-row scales, F, K, G,
    L float32 (the library quantizes every row with its own power-of-two
    scale), or, with fscale_x / fscale_y (float32, N and M), uint8 e4m3 bytes
    quantized by the caller. "side": one power-of-two scale per side (float32
    factors; the faster FP8 kernel)."""
    if fp8 is None:
        fp8 = False
    if fp8 not in (False, True, "rows", "side"):
        raise ValueError("fp8 must be False / None, True / 'rows' or 'side'")
    lib = load()
    N, d = _shape(F)
    M, d2 = _shape(G)
    if _shape(K) != (N, d) or _shape(L) != (M, d2) or d != d2:
        raise ValueError("F, K must be N x d and G, L must be M x d")
    if fscale_x is not None or fscale_y is not None:
        if fp8 not in (True, "rows") or fscale_x is None or fscale_y is None:
            raise ValueError("fscale_x and fscale_y come together, with per-row fp8")
        if not all(_is_bytes(x) for x in (F, K, G, L)):
            raise TypeError("caller-scaled fp8 markets take uint8 e4m3 bytes")
        if _shape(fscale_x) != (N,) or _shape(fscale_y) != (M,):
            raise ValueError("fscale_x must have N entries and fscale_y M entries")
        dt = TU_DTYPE_FP8E4M3
    else:
        dt = _dtype_code(F)
        if any(_dtype_code(x) != dt for x in (K, G, L)):
            raise TypeError("F, K, G, L must share one dtype")
        if fp8:
            if dt != TU_DTYPE_FP32:
                raise TypeError("fp8 markets take float32 factors")
            dt = TU_DTYPE_FP8E4M3_SIDE if fp8 == "side" else TU_DTYPE_FP8E4M3
    n = np.ascontiguousarray(n, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    if n.shape != (N,) or m.shape != (M,):
        raise ValueError("n must have N entries and m must have M entries")
    desc = MarketDesc(N=N, M=M, d=d, dtype=dt, path=TU_PATH_FUSED if path == "fused" else TU_PATH_DENSE,
                      F=_ptr(F), K=_ptr(K), G=_ptr(G), L=_ptr(L), bias_x=_ptr(bias_x), bias_y=_ptr(bias_y),
                      n=_ptr(n), m=_ptr(m), sigma=float(sigma), partition=int(partition),
                      stream=_stream_handle(stream), fscale_x=_ptr(fscale_x), fscale_y=_ptr(fscale_y))
    if path not in ("fused", "dense"):
        raise ValueError("path must be 'fused' or 'dense'")
    h = ctypes.c_void_p()
    _check(lib.tu_market_create(ctypes.byref(desc), ctypes.byref(h)), "tu_market_create")
    return h.value


def tu_market_update_factors(h: int, F, K, G, L) -> None:
    _check(load().tu_market_update_factors(h, _ptr(F), _ptr(K), _ptr(G), _ptr(L)), "tu_market_update_factors", h)


def tu_market_update_factors_fp8(h: int, F, K, G, L, fscale_x, fscale_y) -> None:
    _check(load().tu_market_update_factors_fp8(h, _ptr(F), _ptr(K), _ptr(G), _ptr(L), _ptr(fscale_x),
                                               _ptr(fscale_y)), "tu_market_update_factors_fp8", h)


def tu_ipfp_sweep(h: int, nsweeps: int, residual: bool = False) -> Optional[float]:
    r = ctypes.c_double(float("nan"))
    _check(load().tu_ipfp_sweep(h, int(nsweeps), ctypes.byref(r) if residual else None), "tu_ipfp_sweep", h)
    return r.value if residual else None


def tu_ipfp_solve(h: int, tol: float, max_iter: int, warm_start: bool = False) -> dict:
    info = SolveInfo()
    st = load().tu_ipfp_solve(h, float(tol), int(max_iter), int(bool(warm_start)), ctypes.byref(info))
    if st not in (TU_OK, TU_ERR_NOT_CONVERGED):
        _check(st, "tu_ipfp_solve", h)
    return dict(status=st, converged=st == TU_OK, sweeps=info.sweeps, residual_inf=info.residual_inf,
                residual_l1=info.residual_l1, match_count=info.match_count)


def tu_ipfp_solve_ranking(h: int, k: int, sample: int, check_every: int, patience: int, max_iter: int,
                          warm_start: bool = False, score_eps: float = 1e-4) -> dict:
    """Sweep until the top-k lists of the sampled users of both sides are unchanged
    (positions separated by more than score_eps in log mu) at `patience`
    consecutive checks, `check_every` sweeps apart."""
    info = SolveInfo()
    st = load().tu_ipfp_solve_ranking(h, int(k), int(sample), int(check_every), int(patience), float(score_eps),
                                      int(max_iter), int(bool(warm_start)), ctypes.byref(info))
    if st not in (TU_OK, TU_ERR_NOT_CONVERGED):
        _check(st, "tu_ipfp_solve_ranking", h)
    return dict(status=st, converged=st == TU_OK, sweeps=info.sweeps, residual_inf=info.residual_inf,
                residual_l1=info.residual_l1, match_count=info.match_count)


def tu_mu_block(h: int, x0: int, nx: int, y0: int, ny: int, out, ld: Optional[int] = None) -> None:
    ld = ny if ld is None else ld
    _check(load().tu_mu_block(h, int(x0), int(nx), int(y0), int(ny), _ptr(out), int(ld)), "tu_mu_block", h)


def tu_topk_partners(h: int, side: int, k: int, row0: int, nrows: int, idx, log_mu=None) -> None:
    _check(load().tu_topk_partners(h, int(side), int(k), int(row0), int(nrows), _ptr(idx), _ptr(log_mu)),
           "tu_topk_partners", h)


def tu_get_potentials(h: int, log_u=None, log_v=None) -> None:
    _check(load().tu_get_potentials(h, _ptr(log_u), _ptr(log_v)), "tu_get_potentials", h)


def tu_set_potentials(h: int, log_u=None, log_v=None) -> None:
    _check(load().tu_set_potentials(h, _ptr(log_u), _ptr(log_v)), "tu_set_potentials", h)


def tu_get_potentials_f64(h: int, log_u=None, log_v=None) -> None:
    """The FP64 solver state (float64 arrays or tensors, host or device)."""
    _check(load().tu_get_potentials_f64(h, _ptr(log_u), _ptr(log_v)), "tu_get_potentials_f64", h)


def tu_set_potentials_f64(h: int, log_u=None, log_v=None) -> None:
    _check(load().tu_set_potentials_f64(h, _ptr(log_u), _ptr(log_v)), "tu_set_potentials_f64", h)


def tu_get_potentials_range_f64(h: int, side: int, lo: int, hi: int, out) -> None:
    """FP64 log potentials of users [lo, hi) of one side into `out` (hi - lo doubles)."""
    _check(load().tu_get_potentials_range_f64(h, int(side), int(lo), int(hi), _ptr(out)),
           "tu_get_potentials_range_f64", h)


def tu_ipfp_half_sweep_range(h: int, side: int, lo: int, hi: int, residual: bool = False):
    """Half-sweep of side `side` restricted to its users [lo, hi) (one shard of a
    market split across GPUs); with residual, (max |r| / mass, sum |r|) of the
    shard's equations at the entering state."""
    out = (ctypes.c_double * 2)()
    _check(load().tu_ipfp_half_sweep_range(h, int(side), int(lo), int(hi), out if residual else None),
           "tu_ipfp_half_sweep_range", h)
    return (out[0], out[1]) if residual else None


def tu_fused_halfsweep_noalloc(rows: int, cols: int, kp: int, own_packed, partner_packed, own_bias, own_mass,
                               own_log_u_in, partner_bias, partner_log_v, sigma: float, own_log_u_out,
                               residual: bool = False, stream=None) -> Optional[float]:
    """One fused X half-sweep on caller device buffers, without any device
    allocation (for callers whose device memory is fully budgeted or held by
    another allocator). Returns the residual of the entering state when
    ``residual`` is set (the call then synchronises the stream)."""
    r = ctypes.c_double(float("nan"))
    st = load().tu_fused_halfsweep_noalloc(int(rows), int(cols), int(kp), _ptr(own_packed), _ptr(partner_packed),
                                           _ptr(own_bias), _ptr(own_mass), _ptr(own_log_u_in), _ptr(partner_bias),
                                           _ptr(partner_log_v), float(sigma), _ptr(own_log_u_out),
                                           ctypes.byref(r) if residual else None, _stream_handle(stream))
    _check(st, "tu_fused_halfsweep_noalloc")
    return r.value if residual else None


def tu_market_set_relaxation(h: int, omega: float) -> None:
    """omega = 1: plain IPFP; 1 < omega < 2: fixed over-relaxation; 0: automatic in solve."""
    _check(load().tu_market_set_relaxation(h, float(omega)), "tu_market_set_relaxation", h)


def tu_selftest_wait_timeout(limit_seconds: float):
    """(status, seconds waited) of the bounded device wait on a barrier nothing signals; expect TU_ERR_TIMEOUT."""
    w = ctypes.c_double(float("nan"))
    st = load().tu_selftest_wait_timeout(float(limit_seconds), ctypes.byref(w))
    return st, w.value


def tu_set_checked_mode(enable: bool) -> None:
    """Guard bands around the device buffers of markets created afterwards,
    verified when they are freed (also on with TU_CHECKED=1 at load)."""
    load().tu_set_checked_mode(int(bool(enable)))


def tu_guard_violations():
    """(number of buffers found written outside their bounds, description of the latest)."""
    buf = ctypes.create_string_buffer(256)
    n = load().tu_guard_violations(buf, len(buf))
    return int(n), buf.value.decode()


def tu_market_set_small_tiles(h: int, mode) -> None:
    """Own-tile height: 0 / False 256-row tiles; 1 / True (default) 128-row tiles for markets whose
    256-row tiles leave SMs idle; 2 always 128-row tiles."""
    _check(load().tu_market_set_small_tiles(h, int(mode)), "tu_market_set_small_tiles", h)


def tu_market_set_split(h: int, split: int) -> None:
    """Partner split of the fused half-sweep (1..8 partner ranges per own tile)."""
    _check(load().tu_market_set_split(h, int(split)), "tu_market_set_split", h)


def tu_market_set_partner_blocks(h: int, blocks: int) -> None:
    """Partner blocks (1..8), streamed one after another by all CTAs so that each stays in L2."""
    _check(load().tu_market_set_partner_blocks(h, int(blocks)), "tu_market_set_partner_blocks", h)


def tu_market_get_shape(h: int) -> tuple:
    """(own-tile mode, partner split; -b for b partner blocks) of a market."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().tu_market_get_shape(h, ctypes.byref(a), ctypes.byref(b)), "tu_market_get_shape", h)
    return a.value, b.value


def tu_market_autotune(h: int, reps: int = 3) -> dict:
    """Time the candidate launch shapes on this market, keep the fastest and cache it by shape."""
    info = TuneInfo()
    _check(load().tu_market_autotune(h, int(reps), ctypes.byref(info)), "tu_market_autotune", h)
    return dict(small_tiles=info.small_tiles, split=info.split, ms=info.ms, ms_default=info.ms_default,
                candidates=info.candidates)


def tu_autotune_cache_save(path: str) -> None:
    _check(load().tu_autotune_cache_save(os.fsencode(path)), "tu_autotune_cache_save")


def tu_autotune_cache_load(path: str) -> None:
    _check(load().tu_autotune_cache_load(os.fsencode(path)), "tu_autotune_cache_load")


def tu_autotune_cache_clear() -> None:
    load().tu_autotune_cache_clear()


def tu_relax_schedule(omega: float, tol: float, done, residual) -> np.ndarray:
    """The factors the solve's relaxation controller (setting ``omega``) sets
    after observing residual[i] at done[i] sweeps (host-only, no GPU)."""
    d = np.ascontiguousarray(done, dtype=np.int32)
    r = np.ascontiguousarray(residual, dtype=np.float64)
    if d.shape != r.shape or d.ndim != 1:
        raise ValueError("done and residual must be 1-D arrays of one length")
    out = np.empty(len(d), np.float64)
    st = load().tu_relax_schedule(float(omega), float(tol), d.ctypes.data, r.ctypes.data, len(d), out.ctypes.data)
    _check(st, "tu_relax_schedule")
    return out


def tu_market_set_translation(h: int, enable: bool) -> None:
    """Translation step before every half-sweep of a sweep (default on; same
    fixed point): off gives Eq. iteration exactly."""
    _check(load().tu_market_set_translation(h, int(bool(enable))), "tu_market_set_translation", h)


def tu_market_use_graphs(h: int, enable: bool) -> None:
    """Replay captured CUDA graphs for blocks of sweeps (default), or launch directly (multi-threaded callers)."""
    _check(load().tu_market_use_graphs(h, int(bool(enable))), "tu_market_use_graphs", h)


def tu_market_relax_update(h: int, tol: float) -> None:
    """Automatic relaxation of asynchronous sweeps: feed the last completed block's residual (non-blocking)."""
    _check(load().tu_market_relax_update(h, float(tol)), "tu_market_relax_update", h)


def tu_market_query(h: int):
    """Non-blocking: (idle, residual of the state entering the last sweep,
    match count, sweeps completed); the last three are None while busy."""
    idle = ctypes.c_int(0)
    res = ctypes.c_double(float("nan"))
    match = ctypes.c_double(float("nan"))
    sweeps = ctypes.c_int64(0)
    _check(load().tu_market_query(h, ctypes.byref(idle), ctypes.byref(res), ctypes.byref(match),
                                  ctypes.byref(sweeps)), "tu_market_query", h)
    if not idle.value:
        return False, None, None, None
    return True, res.value, match.value, sweeps.value


def tu_market_footprint(N: int, M: int, d: int, path: str = "fused") -> int:
    """Device bytes a market of this shape holds (admission control)."""
    return int(load().tu_market_footprint(int(N), int(M), int(d), TU_PATH_FUSED if path == "fused" else TU_PATH_DENSE))


def tu_profile_enable(h: int, enable: bool = True) -> None:
    _check(load().tu_profile_enable(h, int(bool(enable))), "tu_profile_enable", h)


def tu_profile_read(h: int):
    """(summed milliseconds, number of timed passes) since the last read."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(load().tu_profile_read(h, ctypes.byref(ms), ctypes.byref(n)), "tu_profile_read", h)
    return ms.value, n.value


def tu_market_destroy(h: int) -> None:
    if h:
        load().tu_market_destroy(h)


def tu_batch_create(handles, stream=None) -> int:
    """Group market handles (fused path, same packed width) into one batch."""
    arr = (ctypes.c_void_p * len(handles))(*[ctypes.c_void_p(h) for h in handles])
    out = ctypes.c_void_p()
    _check(load().tu_batch_create(arr, len(handles), _stream_handle(stream), ctypes.byref(out)), "tu_batch_create")
    return out.value


def tu_batch_sweep(h: int, nsweeps: int, count: int, residual: bool = False):
    """nsweeps sweeps of every market; with residual, a float64 array of count
    per-market residuals of the returned state."""
    r = np.full(count, np.nan, dtype=np.float64) if residual else None
    st = load().tu_batch_sweep(h, int(nsweeps), r.ctypes.data if residual else None)
    _check(st, "tu_batch_sweep", h, batch=True)
    return r


def tu_batch_solve(h: int, tol: float, max_iter: int, count: int, warm_start: bool = False):
    """(overall status, list of per-market dicts as tu_ipfp_solve returns)."""
    infos = (SolveInfo * count)()
    st = load().tu_batch_solve(h, float(tol), int(max_iter), int(bool(warm_start)), infos)
    if st not in (TU_OK, TU_ERR_NOT_CONVERGED, TU_ERR_NONFINITE):
        _check(st, "tu_batch_solve", h, batch=True)
    out = [dict(status=i.status, converged=i.status == TU_OK, sweeps=i.sweeps, residual_inf=i.residual_inf,
                residual_l1=i.residual_l1, match_count=i.match_count) for i in infos]
    return st, out


def tu_batch_profile_enable(h: int, enable: bool = True) -> None:
    _check(load().tu_batch_profile_enable(h, int(bool(enable))), "tu_batch_profile_enable", h, batch=True)


def tu_batch_profile_read(h: int):
    """(summed milliseconds of the batched tensor-core passes, number of passes) since the last read."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(load().tu_batch_profile_read(h, ctypes.byref(ms), ctypes.byref(n)), "tu_batch_profile_read", h,
           batch=True)
    return ms.value, n.value


def tu_batch_destroy(h: int) -> None:
    if h:
        load().tu_batch_destroy(h)


# ---------------------------------------------------------------------------
# convenience object
# ---------------------------------------------------------------------------

class Market:
    """Owning wrapper of a market handle (torch CUDA tensors for outputs)."""

    def __init__(self, F, K, G, L, n, m, sigma, *, bias_x=None, bias_y=None, path="fused", partition=0,
                 stream=None, device="cuda", fp8=False, fscale_x=None, fscale_y=None):
        self.N, self.d = _shape(F)
        self.M = _shape(G)[0]
        self.device = device
        self.stream = stream
        self.handle = tu_market_create(F, K, G, L, n, m, sigma, bias_x=bias_x, bias_y=bias_y, path=path,
                                       partition=partition, stream=stream, fp8=fp8, fscale_x=fscale_x,
                                       fscale_y=fscale_y)

    def sweep(self, nsweeps: int, residual: bool = False):
        return tu_ipfp_sweep(self.handle, nsweeps, residual)

    def solve(self, tol: float, max_iter: int, warm_start: bool = False) -> dict:
        return tu_ipfp_solve(self.handle, tol, max_iter, warm_start)

    def solve_ranking(self, k: int = 10, sample: int = 4096, check_every: int = 5, patience: int = 3,
                      max_iter: int = 10000, warm_start: bool = False, score_eps: float = 1e-4) -> dict:
        return tu_ipfp_solve_ranking(self.handle, k, sample, check_every, patience, max_iter, warm_start, score_eps)

    def set_relaxation(self, omega: float) -> None:
        tu_market_set_relaxation(self.handle, omega)

    def set_translation(self, enable: bool) -> None:
        tu_market_set_translation(self.handle, enable)

    def potentials(self):
        import torch
        lu = torch.empty(self.N, dtype=torch.float32, device=self.device)
        lv = torch.empty(self.M, dtype=torch.float32, device=self.device)
        tu_get_potentials(self.handle, lu, lv)
        self._sync()
        return lu, lv

    def set_potentials(self, log_u=None, log_v=None):
        tu_set_potentials(self.handle, log_u, log_v)

    def potentials64(self):
        """The FP64 state as host numpy arrays (log u, log v)."""
        lu = np.empty(self.N, np.float64)
        lv = np.empty(self.M, np.float64)
        tu_get_potentials_f64(self.handle, lu, lv)
        return lu, lv

    def update_factors(self, F, K, G, L):
        tu_market_update_factors(self.handle, F, K, G, L)

    def mu_block(self, x0=0, nx=None, y0=0, ny=None):
        import torch
        nx = self.N - x0 if nx is None else nx
        ny = self.M - y0 if ny is None else ny
        out = torch.empty((nx, ny), dtype=torch.float32, device=self.device)
        tu_mu_block(self.handle, x0, nx, y0, ny, out, ny)
        self._sync()
        return out

    def topk(self, side: int, k: int, row0: int = 0, nrows: Optional[int] = None):
        import torch
        rows = self.N if side == 0 else self.M
        nrows = rows - row0 if nrows is None else nrows
        idx = torch.empty((nrows, k), dtype=torch.int32, device=self.device)
        lm = torch.empty((nrows, k), dtype=torch.float32, device=self.device)
        tu_topk_partners(self.handle, side, k, row0, nrows, idx, lm)
        self._sync()
        return idx, lm

    def _sync(self):
        import torch
        if self.stream is not None:
            self.stream.synchronize()
        else:
            torch.cuda.synchronize()

    def close(self):
        if getattr(self, "handle", None):
            tu_market_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Owning wrapper of a batch handle over :class:`Market` objects (the
    markets must outlive the batch; it keeps references to them)."""

    def __init__(self, markets, stream=None):
        self.markets = list(markets)
        self.stream = stream
        self.handle = tu_batch_create([mk.handle for mk in self.markets], stream=stream)

    def sweep(self, nsweeps: int, residual: bool = False):
        return tu_batch_sweep(self.handle, nsweeps, len(self.markets), residual)

    def solve(self, tol: float, max_iter: int, warm_start: bool = False):
        return tu_batch_solve(self.handle, tol, max_iter, len(self.markets), warm_start)

    def profile(self, enable: bool = True) -> None:
        tu_batch_profile_enable(self.handle, enable)

    def profile_read(self):
        return tu_batch_profile_read(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            tu_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def from_synth(mk, path: str = "fused", device: str = "cuda", stream=None, partition: int = 0,
               fp8=False) -> Market:
    """Create a :class:`Market` on the device from a ``synth.Market`` (fp8:
    True / "rows" or "side", its float32 factors, quantized by the library to
    e4m3 with per-row or per-side scales)."""
    import torch

    def dev(a):
        if a is None:
            return None
        if mk.dtype == "bf16" and a.ndim == 2 and not fp8:
            bits = (np.ascontiguousarray(a, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)
            return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).to(device)
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)

    F, K, G, L = (dev(x) for x in (mk.F, mk.K, mk.G, mk.L))
    bx, by = dev(mk.bias_x), dev(mk.bias_y)
    torch.cuda.synchronize()
    return Market(F, K, G, L, mk.n, mk.m, mk.sigma, bias_x=bx, bias_y=by, path=path, partition=partition,
                  stream=stream, device=device, fp8=fp8)
