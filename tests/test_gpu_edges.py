"""Edge cases on the GPU: the largest N, the full DFT (J = Z_N), empty
batches, the smallest supports."""
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


@pytest.mark.parametrize("s", [5, 13])
@pytest.mark.parametrize("prec", [0, 1])
def test_largest_N(s, prec):
    # N = 2^62 (the largest the library accepts): N/k = 2^(62-s) folded into the
    # last stage, twiddle residues up to 61 bits
    if prec == 1 and s > 12:
        pytest.skip("complex128 at s = 5 only")
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    M = 62
    rng = np.random.default_rng(6200 + s)
    piv = np.sort(rng.choice(np.arange(M), size=s, replace=False))
    J = W.homogeneous_support(M, piv, rng)
    plan = Plan(M, J, prec)
    Jc = O.canonical_support_by_key(J, piv)
    C = W.complex_gaussian((2, J.size), rng)
    F = O.synthesize_levels(M, piv, Jc, C)
    np_dt = np.complex64 if prec == 0 else np.complex128
    x = torch.from_numpy(F.astype(np_dt)).cuda()
    y = plan.execute_strided(x)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    got = y.cpu().numpy().astype(np.complex128)
    ref = O.transform_levels(M, piv, Jc, x.cpu().numpy().astype(np.complex128))
    tol = 1e-5 if prec == 0 else 1e-12
    assert rel_l2(got, ref) < tol and rel_l2(got, C) < (2e-6 if prec == 0 else 1e-11)


@pytest.mark.parametrize("M", [10, 12, 14])
def test_full_support_is_the_dft(M):
    # J = Z_N: pivots 0..M-1, the transform is the N-point DFT of the samples
    # taken in sample order (compared with a library FFT)
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    N = 1 << M
    plan = Plan(M, np.arange(N, dtype=np.uint64), 0)
    I = plan.sample_indices.astype(np.int64)
    Jc = plan.support_order.astype(np.int64)
    rng = np.random.default_rng(M)
    f = W.complex_gaussian((3, N), rng)
    x = torch.from_numpy(np.ascontiguousarray(f[:, I].astype(np.complex64))).cuda()
    y = plan.execute_strided(x).cpu().numpy().astype(np.complex128)
    ref = np.fft.fft(f, axis=1)[:, Jc]
    assert rel_l2(y, ref) < 1e-5


def test_empty_batches_are_no_ops():
    torch = _torch()
    from paper_2211_15299_gb300 import Plan, Sas, _native as N
    rng = np.random.default_rng(3)
    piv = W.random_pivots(16, 8, rng)
    plan = Plan(16, W.homogeneous_support(16, piv, rng), 0)
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda")
    N.sdft_execute_strided(plan.handle, 0, buf, buf, None)
    N.sdft_synthesize_strided(plan.handle, 0, buf, buf, None)
    sas = Sas(10, [0, 512, 1, 6, 7], "c64")
    N.sdft_sas_execute(sas.handle, 0, buf, buf, buf[8:], None)
    torch.cuda.synchronize()
    assert plan.device_status() == 0 and torch.count_nonzero(buf) == 0


@pytest.mark.parametrize("J", [[5], [3, 7], [0, 1, 2]])
def test_smallest_supports_through_sas(J):
    torch = _torch()
    from paper_2211_15299_gb300 import Sas
    M = 4
    p = Sas(M, J, "c128")
    rng = np.random.default_rng(len(J))
    c = W.complex_gaussian(len(J), rng)
    order = [int(j) for j in p.support_order]
    F = O.sas_samples_direct(M, order, c, p.sample_indices)
    y = p.execute(torch.from_numpy(F.reshape(1, -1)).cuda())
    torch.cuda.synchronize()
    assert rel_l2(y[0].cpu().numpy(), c) < 1e-12 * max(1.0, p.max_cond)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("s", [5, 6, 7, 8, 9, 10])
def test_warp_path_and_tile_path_agree_bitwise(s, prec):
    """Small batches (at most 2^14 values) of 2^5..2^10-point transforms run one
    warp per instance; larger ones the TMA-fed tile kernel. Both apply the same
    butterflies in the same stage order, so the first instances agree bit for bit,
    and both match the oracle."""
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(6500 + 10 * s + prec)
    M = s + 6
    piv = np.sort(rng.choice(np.arange(M), size=s, replace=False))
    J = W.homogeneous_support(M, piv, rng)
    plan = Plan(M, J, prec)
    k = plan.k
    small = (1 << 14) // k                       # the warp path's largest batch
    big = small + 3                              # tile path
    Jc = O.canonical_support_by_key(J, piv)
    C = W.complex_gaussian((big, k), rng)
    F = O.synthesize_levels(M, piv, Jc, C).astype(np.complex64 if prec == 0 else np.complex128)
    x = torch.from_numpy(F).cuda()
    y_tile = plan.execute_strided(x)
    y_warp = plan.execute_strided(x[:small].contiguous())
    y_one = plan.execute(x[0].contiguous())
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    assert torch.equal(y_warp, y_tile[:small])
    assert torch.equal(y_one, y_tile[0])
    tol = 1e-5 if prec == 0 else 1e-12
    assert rel_l2(y_warp.cpu().numpy().astype(np.complex128), C[:small]) < tol


def test_largest_k():
    """k = 2^28 (the largest the library accepts), complex64, one instance: three
    levels of butterflies. Synthesis then transform returns the coefficients;
    Parseval holds; two coefficients match the oracle's closed form."""
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    M, s = 40, 28
    rng = np.random.default_rng(6600)
    piv = np.sort(rng.choice(np.arange(M), size=s, replace=False))
    J = W.homogeneous_support(M, piv, rng)
    plan = Plan(M, J, 0)
    assert len(plan.pivots) == s
    g = torch.Generator(device="cuda")
    g.manual_seed(66)
    C = torch.randn(1 << s, dtype=torch.complex64, device="cuda", generator=g)
    f = plan.synthesize(C)
    y = plan.execute_strided(f)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    c128 = C.to(torch.complex128)
    assert float(torch.linalg.vector_norm(y.to(torch.complex128) - c128) / torch.linalg.vector_norm(c128)) < 1e-5
    fn = float(torch.linalg.vector_norm(f.to(torch.complex128)))
    yn = float(torch.linalg.vector_norm(y.to(torch.complex128)))
    assert abs(yn - fn * (1 << M) / np.sqrt(1 << s)) / yn < 1e-5
    del C
    # two support elements: canonical position t = sum_q bit_{r_q}(j) 2^q, value by
    # the closed form over the oracle's sample set
    I = O.sample_set(M, piv)
    f_h = f.cpu().numpy().astype(np.complex128)
    y_h = y.cpu().numpy()
    js = [int(J[i]) for i in rng.choice(J.size, size=2, replace=False)]
    ts = [sum(((j >> int(r)) & 1) << q for q, r in enumerate(piv)) for j in js]
    spot = O.coefficients_at(M, np.asarray(js, dtype=np.uint64), I, f_h)
    scale = np.linalg.norm(y_h.astype(np.complex128)) / np.sqrt(1 << s)
    assert np.abs(y_h[ts] - spot).max() / scale < 1e-4
