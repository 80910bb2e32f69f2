"""The allocation-free batch entry point (sdft_batch_execute_noalloc).

It serves callers that must not allocate device memory while they run, such
as a serving loop working inside a device-memory budget reserved at start-up:
the batch is built beforehand and the call draws its dependency counters from
an array built into the library. This file is collected last on purpose, so a
run that stops at its first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_batch_execute_twice():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2211_15299_gb300 import Batch, Plan, _native as N
    rng = np.random.default_rng(777)
    # uneven instances, several with two or three levels so the counters are used
    sizes = [21, 16, 14, 13, 12, 9, 5, 3, 0, 15, 13]
    insts = []
    for s in sizes:
        M = max(s, 1) + int(rng.integers(0, 6))
        piv = W.random_pivots(M, s, rng)
        insts.append(W.Instance(M, piv, W.homogeneous_support(M, piv, rng)))
    plans = [Plan(i.M, i.J, 0) for i in insts]
    b = Batch(plans)
    assert b.stats()[1] > 0
    x = torch.randn(b.total, dtype=torch.complex64, device="cuda")
    ref = torch.empty_like(x)
    N.sdft_batch_execute(b.handle, x, ref, torch.cuda.current_stream().cuda_stream)
    for _ in range(2):   # two calls in a row share the built-in counter array
        out = torch.full_like(x, float("nan"))
        N.sdft_batch_execute_noalloc(b.handle, x, out, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert b.device_status() == 0
        err = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
        assert err < 1e-6, err
