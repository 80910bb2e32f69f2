"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle.

Inputs are seeded supports and coefficients from `workloads`; samples come
from the oracle's synthesis; expected values from the oracle only. Tolerances:
relative L2 <= 1e-5 for the complex64 path and <= 1e-12 for complex128.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _run(plan, F):
    """Samples F (B, k) complex128 -> GPU coefficients (B, k) complex128."""
    torch = _torch()
    np_dt = np.complex64 if plan.prec == 0 else np.complex128
    x = torch.from_numpy(np.ascontiguousarray(F.astype(np_dt))).cuda()
    y = plan.execute_strided(x)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return y.cpu().numpy().astype(np.complex128), F.astype(np_dt).astype(np.complex128)


def _case(M, s, batch, rng, prec, coeffs="gauss"):
    from paper_2211_15299_gb300 import Plan
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    plan = Plan(M, J, prec)
    Jc = O.canonical_support_by_key(J, piv)
    assert np.array_equal(plan.support_order, Jc)
    assert np.array_equal(plan.sample_indices, O.sample_set(M, piv))
    C = W.complex_gaussian((batch, J.size), rng) if coeffs == "gauss" else W.log_uniform_coeffs((batch, J.size), rng)
    F = O.synthesize_levels(M, piv, Jc, C)
    return plan, piv, Jc, C, F


@pytest.mark.parametrize("prec", [0, 1])
def test_brute_force_n16_k4(prec):
    from paper_2211_15299_gb300 import Plan
    rng = W.rng_for(1, 7)
    for trial in range(8):
        piv = W.random_pivots(4, 2, rng)
        J = W.homogeneous_support(4, piv, rng)
        plan = Plan(4, J, prec)
        Jc = O.canonical_support(J, piv)
        I = O.sample_set(4, piv)
        c = W.complex_gaussian(4, rng)
        f = O.brute_force_samples(4, Jc, c, I)
        got, f_in = _run(plan, f[None, :])
        assert rel_l2(got[0], c) < TOL[prec] * 10
        assert rel_l2(got[0], O.solve(4, Jc, I, f_in[0])) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_config1_single_instance(prec):
    from paper_2211_15299_gb300 import Plan
    inst = W.workload_single()
    plan = Plan(inst.M, inst.J, prec)
    Jc = O.canonical_support(inst.J, inst.pivots)
    I = O.sample_set(inst.M, inst.pivots)
    cmap = dict(zip([int(j) for j in inst.J], inst.coeffs))
    c = np.array([cmap[int(j)] for j in Jc])
    f = O.synthesize(inst.M, Jc, c, I)
    got, f_in = _run(plan, f[None, :])
    ref = O.solve(inst.M, Jc, I, f_in[0])
    assert rel_l2(got[0], ref) < TOL[prec]
    assert rel_l2(got[0], c) < max(TOL[prec], 1e-6 if prec == 0 else 0)


# (M, s, batch): k from 1 to 2^16 (complex64) / 2^15 (complex128); batches chosen so
# the packed length leaves a ragged last tile; s > 12 (resp. 11) runs two levels.
SIZES = [(1, 0, 5), (3, 1, 7), (6, 2, 9), (8, 3, 33), (9, 4, 65), (10, 5, 37), (12, 6, 19),
         (14, 7, 37), (11, 8, 5), (20, 9, 11), (16, 10, 3), (24, 11, 5), (13, 12, 6), (18, 13, 3),
         (22, 14, 2), (26, 15, 2), (17, 16, 2)]


@pytest.mark.parametrize("M,s,batch", SIZES)
@pytest.mark.parametrize("prec", [0, 1])
def test_sizes_against_oracle(M, s, batch, prec):
    rng = np.random.default_rng(1000 * s + M + 17 * prec)
    plan, piv, Jc, C, F = _case(M, s, batch, rng, prec)
    got, f_in = _run(plan, F)
    ref = O.transform_levels(M, piv, Jc, f_in)
    for b in range(batch):
        assert rel_l2(got[b], ref[b]) < TOL[prec], b
    assert rel_l2(got, C) < (2e-6 if prec == 0 else 1e-12)


@pytest.mark.parametrize("s", [20, 21])
def test_three_levels_complex64(s):
    # s = 21 adds a third level (bits [20, 21)) after the two 4096-wide ones.
    rng = np.random.default_rng(4242 + s)
    plan, piv, Jc, C, F = _case(s + 3, s, 2, rng, 0)
    got, f_in = _run(plan, F)
    ref = O.transform_levels(s + 3, piv, Jc, f_in)
    assert rel_l2(got, ref) < TOL[0]


@pytest.mark.parametrize("s", [19, 20])
def test_three_levels_complex128(s):
    # complex128 tiles hold 2^11 values and later levels 8 stage bits: s = 19
    # runs levels [0, 11) and [11, 19); s = 20 adds a third level [19, 20).
    # The FP64 pipe against the oracle at 1e-12, element by element.
    rng = np.random.default_rng(5252 + s)
    plan, piv, Jc, C, F = _case(s + 2, s, 1, rng, 1)
    got, f_in = _run(plan, F)
    ref = O.transform_levels(s + 2, piv, Jc, f_in)
    assert rel_l2(got, ref) < TOL[1]
    assert rel_l2(got, C) < TOL[1]


def test_inplace():
    torch = _torch()
    rng = np.random.default_rng(77)
    plan, piv, Jc, C, F = _case(20, 14, 3, rng, 0)
    x = torch.from_numpy(F.astype(np.complex64)).cuda()
    ref = plan.execute_strided(x.clone())
    plan.execute_strided(x, x)
    torch.cuda.synchronize()
    assert torch.equal(x, ref)


def test_misaligned_buffers_rejected():
    torch = _torch()
    from paper_2211_15299_gb300 import Plan, SdftError, _native as N
    plan = Plan(10, list(range(32)), 0)
    buf = torch.zeros(2 * 64 + 8, dtype=torch.float32, device="cuda")
    with pytest.raises(SdftError) as ei:
        N.sdft_execute(plan.handle, buf.data_ptr() + 8, buf.data_ptr() + 8 + 512, None)
    assert ei.value.name == "SDFT_ERR_ARG"
    with pytest.raises(SdftError) as ei:      # partial overlap
        N.sdft_execute(plan.handle, buf.data_ptr(), buf.data_ptr() + 16, None)
    assert ei.value.name == "SDFT_ERR_ARG"


@pytest.mark.parametrize("prec", [0, 1])
def test_config2_full_size(prec):
    """N = 2^20, k = 2^12, batch 4096, one shared plan, log-uniform magnitudes."""
    from paper_2211_15299_gb300 import Plan
    inst, C = W.workload_shared()
    plan = Plan(inst.M, inst.J, prec)
    Jc = O.canonical_support_by_key(inst.J, inst.pivots)
    F = O.synthesize_levels(inst.M, inst.pivots, Jc, C)
    got, f_in = _run(plan, F)
    per = np.linalg.norm(got - C, axis=1) / np.linalg.norm(C, axis=1)
    assert per.max() < (1e-5 if prec == 0 else 1e-12)
    # spot checks: single coefficients by the closed form on the same rounded input
    rng = np.random.default_rng(5)
    I = O.sample_set(inst.M, inst.pivots)
    for b in rng.choice(C.shape[0], size=4, replace=False):
        idx = rng.choice(C.shape[1], size=16, replace=False)
        spot = O.coefficients_at(inst.M, Jc[idx], I, f_in[b])
        err = np.abs(got[b, idx] - spot).max() / np.linalg.norm(C[b]) * np.sqrt(C.shape[1])
        assert err < TOL[prec]


@pytest.mark.parametrize("contiguous", [True, False])
def test_config3_full_size(contiguous):
    """N = 2^30, k = 2^20, batch 64, complex64 (two levels of butterflies): every
    instance synthesised by the oracle from seeded coefficients and compared
    element by element with them; four against the oracle's transform of the
    same rounded samples; Parseval for all; closed-form spot checks."""
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    inst, _ = W.workload_large(contiguous=contiguous, coeffs=False)
    rng = W.rng_for(3, 100 + int(contiguous))
    plan = Plan(inst.M, inst.J, 0)
    Jc = O.canonical_support_by_key(inst.J, inst.pivots)
    B, k = 64, inst.k
    C = W.complex_gaussian((B, k), rng)
    F = np.empty((B, k), dtype=np.complex64)
    for b0 in range(0, B, 16):                      # the oracle's synthesis, 16 at a time
        F[b0:b0 + 16] = O.synthesize_levels(inst.M, inst.pivots, Jc, C[b0:b0 + 16])
    # the synthesis itself at a few sample points by the direct sum
    I = O.sample_set(inst.M, inst.pivots)
    pts = rng.choice(k, size=32, replace=False)
    direct = O.brute_force_samples(inst.M, Jc, C[5], I[pts])
    assert rel_l2(F[5, pts], direct) < 1e-6
    x = torch.from_numpy(F).cuda()
    y = plan.execute_strided(x)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    got = y.cpu().numpy()
    for b in range(B):                              # every instance against its coefficients
        assert rel_l2(got[b], C[b]) < 1e-5, b
    for b in (0, 21, 42, 63):                       # element by element against the oracle
        ref = O.transform_levels(inst.M, inst.pivots, Jc, F[b:b + 1].astype(np.complex128))[0]
        assert rel_l2(got[b], ref) < TOL[0], b
    # Parseval for every instance: ||c||^2 = (N^2 / k) ||f||^2 (F(J, I) is sqrt(k)-scaled unitary)
    fn = torch.linalg.vector_norm(x.to(torch.complex128), dim=1).cpu().numpy()
    cn = torch.linalg.vector_norm(y.to(torch.complex128), dim=1).cpu().numpy()
    assert np.allclose(cn, fn * (1 << inst.M) / np.sqrt(k), rtol=1e-5)
    # spot checks by the closed form on the same rounded samples
    for b in (17, 63):
        idx = rng.choice(k, size=8, replace=False)
        spot = O.coefficients_at(inst.M, Jc[idx], I, F[b].astype(np.complex128))
        row = got[b].astype(np.complex128)
        assert np.abs(row[idx] - spot).max() / (np.linalg.norm(row) / np.sqrt(k)) < 1e-5


def test_config4_full_uneven_workload():
    """The 10,000-instance uneven workload (each instance its own support, N from
    2^12 to 2^24, k from 2^4 to 2^16) in one batch launch, every instance against
    the oracle's transform of the same rounded samples at 1e-5."""
    torch = _torch()
    from paper_2211_15299_gb300 import Batch, Plan
    insts = W.workload_uneven(count=10000)
    plans = [Plan(i.M, i.J, 0) for i in insts]
    b = Batch(plans)
    rng = W.rng_for(4, 31)
    x = torch.from_numpy(W.complex_gaussian(b.total, rng).astype(np.complex64)).cuda()
    y = b.execute(x)
    torch.cuda.synchronize()
    assert b.device_status() == 0
    xs, ys = x.cpu().numpy(), y.cpu().numpy()
    worst = 0.0
    for i, (inst, p) in enumerate(zip(insts, plans)):
        o, kk = int(b.offsets[i]), p.k
        Jc = O.canonical_support_by_key(inst.J, inst.pivots)
        ref = O.transform_levels(inst.M, inst.pivots, Jc, xs[o:o + kk][None].astype(np.complex128))[0]
        err = rel_l2(ys[o:o + kk], ref)
        worst = max(worst, err)
        assert err < TOL[0], (i, inst.M, inst.s, err)
    assert worst > 0.0


@pytest.mark.parametrize("prec", [0, 1])
def test_user_order(prec):
    """The optional reordering into the caller's order of J: coefficient u is the
    one of J[u] (J shuffled before planning), against the oracle."""
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(9400 + prec)
    M, s, B = 18, 13, 3
    piv = np.sort(rng.choice(np.arange(M), size=s, replace=False))
    J = W.homogeneous_support(M, piv, rng)
    J_user = rng.permutation(J)
    plan = Plan(M, J_user, prec, user_order=True)
    assert plan.device_bytes == Plan(M, J_user, prec).device_bytes + 4 * plan.k   # the positions
    Jc = O.canonical_support_by_key(J, piv)
    C = W.complex_gaussian((B, plan.k), rng)
    F = O.synthesize_levels(M, piv, Jc, C)
    dt = np.complex64 if prec == 0 else np.complex128
    y = plan.execute_strided(torch.from_numpy(F.astype(dt)).cuda())
    yu = plan.to_user_order(y)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    where = {int(j): t for t, j in enumerate(Jc)}
    C_user = C[:, [where[int(j)] for j in J_user]]
    assert rel_l2(yu.cpu().numpy().astype(np.complex128), C_user) < (1e-5 if prec == 0 else 1e-12)
    # plans without the flag refuse the call
    from paper_2211_15299_gb300 import SdftError
    with pytest.raises(SdftError):
        Plan(M, J_user, prec).to_user_order(y)
