import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpu_lib():
    """The C-ABI library, loaded through the Python binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_19214_gb300 as tu
    from paper_2411_19214_gb300 import build as tb
    tb.build()
    tu.load()
    return tu


@pytest.fixture(autouse=True)
def _guard_bands(request):
    """After every GPU test: no market buffer was written outside its bounds.
    The library counts guard-band violations of buffers it frees; the bands
    exist when checked mode is on (TU_CHECKED=1 when the library is loaded),
    so `TU_CHECKED=1 pytest -m gpu` runs the whole suite with them."""
    if request.node.get_closest_marker("gpu") is None:
        yield
        return
    import paper_2411_19214_gb300 as tu
    before = tu.tu_guard_violations()[0] if tu._lib is not None else 0
    yield
    if tu._lib is not None:
        n, last = tu.tu_guard_violations()
        assert n == before, f"{n - before} buffer(s) written outside their bounds; latest: {last}"
