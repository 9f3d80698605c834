"""The C-ABI library builds, loads and exports every symbol its header declares.

No compute call is made here (no GPU needed): only argument validation that
the library performs before touching CUDA.
"""

import ctypes
import os
import re

import numpy as np
import pytest

import paper_2411_19214_gb300 as tu
from paper_2411_19214_gb300 import build as tb

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


@pytest.fixture(scope="module")
def lib():
    tb.build()
    return tu.load()


def _declared():
    names = set()
    for f in os.listdir(HEADER_DIR):
        if f.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tu_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 11
    for name in declared:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert tu.status_string(0) == "TU_OK"
    assert tu.status_string(4) == "TU_ERR_NOT_CONVERGED"
    assert tu.status_string(7) == "TU_ERR_UNSUPPORTED"
    assert tu.status_string(99) == "TU_ERR_UNKNOWN"


def test_invalid_arguments_rejected_before_cuda(lib):
    F = np.zeros((4, 3), np.float32)
    n = np.ones(4)
    bad = [
        dict(sigma=0.0),
        dict(sigma=-1.0),
        dict(sigma=float("nan")),
    ]
    for kw in bad:
        with pytest.raises(tu.TuError) as e:
            tu.tu_market_create(F, F, F, F, n, n, **kw)
        assert e.value.status == tu.TU_ERR_INVALID_ARG
    # null descriptor / output
    assert lib.tu_market_create(None, None) == tu.TU_ERR_INVALID_ARG
    d = tu.MarketDesc(N=0, M=4, d=3, dtype=1, path=0)
    h = ctypes.c_void_p()
    assert lib.tu_market_create(ctypes.byref(d), ctypes.byref(h)) == tu.TU_ERR_INVALID_ARG
    # the size limits of the header's create contract, each with its status;
    # every one is decided before the library touches CUDA (the pointers are
    # placeholders that are never read)
    ptrs = dict(F=1, K=1, G=1, L=1, n=1, m=1, sigma=1.0)
    limits = [
        (dict(N=(1 << 31) + 1, M=4, d=3, dtype=1, path=1), tu.TU_ERR_INVALID_ARG),
        (dict(N=4, M=(1 << 31) + 1, d=3, dtype=1, path=1), tu.TU_ERR_INVALID_ARG),
        (dict(N=4, M=4, d=4097, dtype=1, path=1), tu.TU_ERR_INVALID_ARG),
        (dict(N=4, M=4, d=3, dtype=4, path=0), tu.TU_ERR_INVALID_ARG),  # unknown dtype
        (dict(N=4, M=4, d=3, dtype=tu.TU_DTYPE_FP8E4M3_SIDE, path=1), tu.TU_ERR_UNSUPPORTED),  # FP8: fused only
        (dict(N=4, M=4, d=3, dtype=tu.TU_DTYPE_FP8E4M3_SIDE, path=0, fscale_x=1, fscale_y=1), tu.TU_ERR_INVALID_ARG),
        (dict(N=4, M=4, d=3, dtype=1, path=2), tu.TU_ERR_INVALID_ARG),  # unknown path
        (dict(N=4, M=4, d=129, dtype=1, path=0), tu.TU_ERR_UNSUPPORTED),  # fused: d <= 128
        (dict(N=4, M=4, d=257, dtype=tu.TU_DTYPE_FP8E4M3, path=0), tu.TU_ERR_UNSUPPORTED),  # FP8: d <= 256
        # caller FP8 scales: both sides, FP8 markets only
        (dict(N=4, M=4, d=3, dtype=tu.TU_DTYPE_FP8E4M3, path=0, fscale_x=1), tu.TU_ERR_INVALID_ARG),
        (dict(N=4, M=4, d=3, dtype=1, path=0, fscale_x=1, fscale_y=1), tu.TU_ERR_INVALID_ARG),
        (dict(N=4, M=4, d=3, dtype=tu.TU_DTYPE_FP8E4M3, path=1), tu.TU_ERR_UNSUPPORTED),  # FP8: fused only
        # dense: A-hat and its transpose, 2 x 4 B x 160,000 x 160,000 = 205 GB > 200 GB
        (dict(N=160_000, M=160_000, d=3, dtype=1, path=1), tu.TU_ERR_UNSUPPORTED),
    ]
    for shape, want in limits:
        d = tu.MarketDesc(**shape, **ptrs)
        assert lib.tu_market_create(ctypes.byref(d), ctypes.byref(h)) == want, shape
    # calls on a null market
    assert lib.tu_ipfp_sweep(None, 1, None) == tu.TU_ERR_INVALID_ARG
    lib.tu_market_destroy(None)
    assert lib.tu_market_last_error(None) == b""


def test_binding_rejects_shape_mismatch(lib):
    F = np.zeros((4, 3), np.float32)
    with pytest.raises(ValueError):
        tu.tu_market_create(F, F, np.zeros((5, 2), np.float32), np.zeros((5, 2), np.float32), np.ones(4),
                            np.ones(5), 1.0)
    with pytest.raises(TypeError):
        tu.tu_market_create(F.astype(np.float64), F, F, F, np.ones(4), np.ones(4), 1.0)


def test_noalloc_and_batch_arguments_rejected_before_cuda(lib):
    """The allocation-free half-sweep and the batch calls decide their
    documented refusals before touching CUDA (placeholder pointers, 16-byte
    aligned, are never read)."""
    INV, UNS = tu.TU_ERR_INVALID_ARG, tu.TU_ERR_UNSUPPORTED
    P = 1 << 20  # a placeholder device address

    def noalloc(rows=100, cols=200, kp=64, own=P, par=P, mass=P, lu_in=P, lv=P, out=P, sigma=0.5):
        return lib.tu_fused_halfsweep_noalloc(rows, cols, kp, own, par, None, mass, lu_in, None, lv, sigma, out,
                                              None, None)

    cases = [
        (dict(rows=0), INV), (dict(cols=0), INV), (dict(sigma=0.0), INV), (dict(sigma=float("inf")), INV),
        (dict(sigma=float("nan")), INV), (dict(own=None), INV), (dict(par=None), INV), (dict(mass=None), INV),
        (dict(lu_in=None), INV), (dict(lv=None), INV), (dict(out=None), INV),
        (dict(rows=65537), UNS), (dict(cols=1048577), UNS), (dict(kp=96), UNS), (dict(kp=256), UNS),
        (dict(own=P + 8), INV), (dict(par=P + 4), INV),  # packed factors must be 16-byte aligned
    ]
    for kw, want in cases:
        assert noalloc(**kw) == want, kw
    V = ctypes.c_void_p
    h = V()
    two_null = (V * 2)(None, None)
    assert lib.tu_batch_create(None, 1, None, ctypes.byref(h)) == INV
    assert lib.tu_batch_create(two_null, 0, None, ctypes.byref(h)) == INV
    assert lib.tu_batch_create(two_null, 65537, None, ctypes.byref(h)) == INV
    assert lib.tu_batch_create(two_null, 2, None, ctypes.byref(h)) == INV  # NULL members
    assert lib.tu_batch_create(two_null, 2, None, None) == INV
    assert lib.tu_batch_sweep(None, 1, None) == INV
    assert lib.tu_batch_solve(None, 1e-6, 10, 0, None) == INV
    assert lib.tu_batch_profile_enable(None, 1) == INV
    assert lib.tu_batch_profile_read(None, None, None) == INV
    lib.tu_batch_destroy(None)
    assert lib.tu_batch_last_error(None) == b""


def test_footprint_counts_the_documented_buffers(lib):
    """tu_market_footprint (pure host arithmetic) holds at least the buffers
    the header names: the packed factors (fused) or A-hat and its transpose
    (dense), and the upload staging; 0 for an invalid shape."""
    for N, M, d in [(1, 1, 1), (1000, 3000, 16), (1_000_000, 1_000_000, 64), (20_000, 10_000, 32)]:
        fused = tu.tu_market_footprint(N, M, d, "fused")
        dense = tu.tu_market_footprint(N, M, d, "dense")
        staging = 2 * max(N, M) * d * 2
        assert fused >= (N + M) * 2 * d * 2 + staging
        assert dense >= 2 * N * M * 4 + staging
        # the per-user state and fixed scratch are O(N + M), a few hundred bytes per user at most
        assert fused - (N + M) * 2 * d * 2 - 2 * max(N, M) * d * 4 <= 300 * (N + M) + (1 << 20)
    assert tu.tu_market_footprint(0, 5, 3, "fused") == 0
    assert tu.tu_market_footprint(5, 5, 0, "dense") == 0


def test_binding_fp8_argument(lib):
    """fp8 = None or False is a BF16/FP32 market, True / "rows" / "side" an
    FP8 one (float32 factors); anything else is refused before the library.
    Without a GPU a well-formed call reaches the library, which answers
    TU_ERR_CUDA (or TU_ERR_UNSUPPORTED for a device it was not built for)."""
    F = np.zeros((4, 3), np.float32)
    for v in (None, False, True, "rows", "side"):
        with pytest.raises(tu.TuError) as e:
            tu.tu_market_create(F, F, F, F, np.ones(4), np.ones(4), 1.0, fp8=v)
        assert e.value.status in (tu.TU_ERR_CUDA, tu.TU_ERR_UNSUPPORTED)
    with pytest.raises(ValueError):
        tu.tu_market_create(F, F, F, F, np.ones(4), np.ones(4), 1.0, fp8="per-tile")
    with pytest.raises(TypeError):
        tu.tu_market_create(F.astype(np.uint16), F.astype(np.uint16), F.astype(np.uint16), F.astype(np.uint16),
                            np.ones(4), np.ones(4), 1.0, fp8=True)


def test_binding_loads_the_library_build_writes():
    """The binding's library path is where build.py puts the library."""
    import paper_2411_19214_gb300 as tu
    from paper_2411_19214_gb300 import build
    assert os.path.realpath(tu.LIB_PATH) == os.path.realpath(build.LIB)
