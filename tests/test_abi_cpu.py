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
        (dict(N=4, M=4, d=3, dtype=3, path=0), tu.TU_ERR_INVALID_ARG),  # unknown dtype
        (dict(N=4, M=4, d=3, dtype=1, path=2), tu.TU_ERR_INVALID_ARG),  # unknown path
        (dict(N=4, M=4, d=65, dtype=1, path=0), tu.TU_ERR_UNSUPPORTED),  # fused: 2d <= 128
        (dict(N=4, M=4, d=65, dtype=tu.TU_DTYPE_FP8E4M3, path=0), tu.TU_ERR_UNSUPPORTED),
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
