"""GPU: transforms on host buffers (sdft_execute_strided_host), chunked and
overlapped, give the same bits as the device path on every chunking."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("prec,s,batch,chunks", [
    (0, 12, 100, (0, 1, 7, 1000)),
    (0, 0, 33, (0, 1, 3)),        # 8-byte instances: chunks rounded up to 16 bytes
    (0, 2, 33, (0, 5)),
    (0, 14, 9, (0, 4)),           # two levels per chunk
    (1, 11, 20, (0, 6)),
])
def test_host_path_matches_device_path(prec, s, batch, chunks):
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(8800 + 10 * s + prec)
    M = s + 5
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    plan = Plan(M, J, prec)
    dt = torch.complex64 if prec == 0 else torch.complex128
    Jc = O.canonical_support_by_key(J, piv)
    C = W.complex_gaussian((batch, plan.k), rng)
    F = O.synthesize_levels(M, piv, Jc, C).astype(np.complex64 if prec == 0 else np.complex128)
    h_in = torch.from_numpy(F.reshape(-1)).pin_memory()
    ref = plan.execute_strided(h_in.cuda()).cpu()
    for chunk in chunks:
        h_out = torch.empty_like(h_in).pin_memory()
        got = plan.execute_host(h_in, h_out, chunk=chunk)
        torch.cuda.current_stream().synchronize()
        assert plan.device_status() == 0
        assert torch.equal(got, ref), chunk
    assert rel_l2(ref.numpy().astype(np.complex128).reshape(batch, -1), C) < (1e-5 if prec == 0 else 1e-12)


def test_host_path_in_place_and_on_a_side_stream():
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(8901)
    M, s, batch = 18, 12, 64
    piv = W.random_pivots(M, s, rng)
    plan = Plan(M, W.homogeneous_support(M, piv, rng), 0)
    x = torch.randn(batch * plan.k, dtype=torch.complex64)
    ref = plan.execute_strided(x.cuda()).cpu()
    h = x.clone().pin_memory()
    side = torch.cuda.Stream()
    d_in = torch.empty(batch * plan.k, dtype=torch.complex64, device="cuda")
    d_out = torch.empty_like(d_in)
    with torch.cuda.stream(side):
        plan.execute_host(h, h, d_in, d_out, chunk=10, stream=side.cuda_stream)   # host buffers in place
    side.synchronize()
    assert torch.equal(h, ref)
    # repeated calls reuse the plan's copy streams and events
    for _ in range(3):
        h2 = x.clone().pin_memory()
        plan.execute_host(h2, h2, d_in, d_out, chunk=16)
        torch.cuda.current_stream().synchronize()
        assert torch.equal(h2, ref)
    assert plan.device_status() == 0


@pytest.mark.parametrize("prec,s,batch", [(0, 12, 40), (0, 15, 6), (1, 11, 10)])
def test_host_synthesis_round_trip(prec, s, batch):
    """synthesize_host equals the device synthesis bit for bit, and host
    transform after host synthesis returns the coefficients."""
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(8950 + s + prec)
    M = s + 4
    piv = W.random_pivots(M, s, rng)
    plan = Plan(M, W.homogeneous_support(M, piv, rng), prec)
    dt = torch.complex64 if prec == 0 else torch.complex128
    C = torch.from_numpy(W.complex_gaussian((batch, plan.k), rng)).to(dt).reshape(-1)
    ref = plan.synthesize(C.cuda()).cpu()
    h_c = C.clone().pin_memory()
    h_f = plan.synthesize_host(h_c, chunk=3)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(h_f, ref)
    back = plan.execute_host(h_f.pin_memory(), chunk=5)
    torch.cuda.current_stream().synchronize()
    assert plan.device_status() == 0
    err = float(torch.linalg.vector_norm((back - C).to(torch.complex128)) / torch.linalg.vector_norm(C.to(torch.complex128)))
    assert err < (1e-5 if prec == 0 else 1e-12)
