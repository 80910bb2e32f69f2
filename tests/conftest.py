import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built extension")
    config.addinivalue_line("markers", "slow: longer CPU test")


def read_golden(name):
    """Lines of a golden fixture, comments and blank lines removed."""
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.strip() for ln in fh if ln.strip() and not ln.lstrip().startswith("#")]


def rel_l2(x, ref):
    import numpy as np
    x = np.asarray(x, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


@pytest.fixture(autouse=True)
def _poison_new_buffers(request, monkeypatch):
    """In GPU tests every buffer made by torch.empty / torch.empty_like (the
    tests' own outputs and the ones the binding allocates) starts as NaN, so a
    coefficient the library never writes cannot pass on stale memory: it makes
    relative errors NaN and torch.equal false."""
    if request.node.get_closest_marker("gpu") is None:
        yield
        return
    import torch
    real_empty, real_empty_like = torch.empty, torch.empty_like

    def _nan(t):
        if t.is_floating_point() or t.is_complex():
            t.fill_(float("nan"))
        return t

    monkeypatch.setattr(torch, "empty", lambda *a, **k: _nan(real_empty(*a, **k)))
    monkeypatch.setattr(torch, "empty_like", lambda *a, **k: _nan(real_empty_like(*a, **k)))
    yield


@pytest.fixture(autouse=True)
def _no_range_check_violations(request):
    """With the debug library (built with SDFT_BOUNDS_CHECK=1) every GPU test
    must end without a range-check violation in any kernel it launched."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    from paper_2211_15299_gb300 import _native as N
    import torch
    torch.cuda.synchronize()
    enabled, count = N.sdft_debug_bounds_violations(clear=True)
    if enabled:
        assert count == 0, f"{count} range-check violations"
