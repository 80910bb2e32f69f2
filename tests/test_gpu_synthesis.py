"""GPU parity of synthesis (samples from coefficients, the inverse of the
transform) against the oracle's FP64 synthesis."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}

SIZES = [(1, 0, 5), (3, 1, 7), (6, 2, 9), (8, 3, 33), (9, 4, 65), (10, 5, 37), (12, 6, 19),
         (14, 7, 37), (11, 8, 5), (20, 9, 11), (16, 10, 3), (24, 11, 5), (13, 12, 6), (18, 13, 3),
         (22, 14, 2), (26, 15, 2), (17, 16, 2), (23, 20, 2), (24, 21, 2)]


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("M,s,batch", SIZES)
@pytest.mark.parametrize("prec", [0, 1])
def test_synthesis_against_oracle(M, s, batch, prec):
    if prec == 1 and s > 15:
        pytest.skip("complex128 sizes capped at 2^15 here")
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(3000 + 7 * s + M + prec)
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    plan = Plan(M, J, prec)
    Jc = O.canonical_support_by_key(J, piv)
    C = W.complex_gaussian((batch, J.size), rng)
    np_dt = np.complex64 if prec == 0 else np.complex128
    c_in = torch.from_numpy(C.astype(np_dt)).cuda()
    f = plan.synthesize(c_in)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    ref = O.synthesize_levels(M, piv, Jc, c_in.cpu().numpy().astype(np.complex128))
    got = f.cpu().numpy().astype(np.complex128)
    for b in range(batch):
        assert rel_l2(got[b], ref[b]) < TOL[prec], b
    # the transform of the synthesised samples returns the coefficients
    back = plan.execute_strided(f).cpu().numpy().astype(np.complex128)
    assert rel_l2(back, C) < 2 * TOL[prec]


def test_synthesis_in_place_and_single_instance():
    torch = _torch()
    from paper_2211_15299_gb300 import Plan, _native as N
    rng = np.random.default_rng(77)
    piv = W.random_pivots(20, 14, rng)
    J = W.homogeneous_support(20, piv, rng)
    plan = Plan(20, J, 0)
    c = torch.from_numpy(W.complex_gaussian((3, J.size), rng).astype(np.complex64)).cuda()
    ref = plan.synthesize(c.clone())
    x = c.clone()
    plan.synthesize(x, x)
    torch.cuda.synchronize()
    assert torch.equal(x, ref)
    one = torch.empty_like(c[0])
    N.sdft_synthesize(plan.handle, c[1], one, None)
    torch.cuda.synchronize()
    assert torch.equal(one, ref[1])


@pytest.mark.parametrize("contiguous", [True, False])
def test_round_trip_at_large_k(contiguous):
    """N = 2^30, k = 2^20, batch 64, complex64: synthesis then transform gives
    the coefficients back; synthesised samples match the direct sum at spots."""
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    inst, _ = W.workload_large(contiguous=contiguous, coeffs=False)
    rng = W.rng_for(3, 300 + int(contiguous))
    plan = Plan(inst.M, inst.J, 0)
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    c = torch.randn((64, inst.k), dtype=torch.complex64, device="cuda", generator=g)
    f = plan.synthesize(c)
    back = plan.execute_strided(f)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    err = torch.linalg.vector_norm((back - c).to(torch.complex128)) / torch.linalg.vector_norm(c.to(torch.complex128))
    assert float(err) < 2e-5
    Jc = O.canonical_support_by_key(inst.J, inst.pivots)
    I = O.sample_set(inst.M, inst.pivots)
    for b in (0, 41):
        cb = c[b].cpu().numpy().astype(np.complex128)
        fb = f[b].cpu().numpy().astype(np.complex128)
        for t in rng.choice(inst.k, size=4, replace=False):
            want = O.synthesize(inst.M, Jc, cb, I[[t]])[0]
            assert abs(fb[t] - want) < 1e-5 * np.linalg.norm(fb) / np.sqrt(inst.k)
